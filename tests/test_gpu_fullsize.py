"""Full-size checks in the launch configuration bench.py times (m = n = 16384, q = 2, reorth).

At this size the oracle cannot compute U, R, V; the checks are properties that
hold at any size: ||A - U R V^T||_F / ||A||_F <= 1e-6 for the mixed path (the
metric's bar), orthogonality, R upper triangular with a nonnegative diagonal,
and ||R||_F = ||A||_F.  Norms of residuals are estimated with Gaussian probe
vectors (E ||M X||_F^2 = k ||M||_F^2), computed in FP64.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _probe_rel(Mx, Ax):
    import torch
    return (torch.linalg.norm(Mx) / torch.linalg.norm(Ax)).item()


def test_mixed_16384_meets_the_reconstruction_bar(B):
    import torch
    from paper_1812_06007_gb300 import workloads as W
    n = 16384
    A = W.test_matrix_torch(n, n, W.sigma_profile("exponential", n, decades=6), device="cuda")
    U, R, V = B.purl_urv_factor(A, 2, True, W.SEED_G, mode=B.PURL_MODE_MIXED_BF16)
    torch.cuda.synchronize()
    assert B.purl_device_status() == B.PURL_OK
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    X = torch.randn(n, 16, generator=g, device="cuda", dtype=torch.float64)
    AX = A @ X
    recon = _probe_rel(AX - U @ (R @ (V.t() @ X)), AX)
    assert recon <= 1e-6, recon
    ou = (torch.linalg.norm(U.t() @ (U @ X) - X) / math.sqrt(16)).item()
    ov = (torch.linalg.norm(V.t() @ (V @ X) - X) / math.sqrt(16)).item()
    assert ou <= 1e-3 and ov <= 1e-3  # Frobenius over n^2 entries: ~3e-9 per entry
    assert torch.count_nonzero(torch.tril(R, -1)).item() == 0
    assert bool((torch.diagonal(R) >= 0).all())
    nA = torch.linalg.norm(A).item()
    assert abs(torch.linalg.norm(R).item() - nA) <= 2e-6 * nA


def test_fp64_4096_meets_its_bar(B):
    import torch
    from paper_1812_06007_gb300 import workloads as W
    n = 4096
    A = W.test_matrix_torch(n, n, W.sigma_profile("exponential", n, decades=6), device="cuda")
    U, R, V = B.purl_urv_factor(A, 2, True, W.SEED_G)
    torch.cuda.synchronize()
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    X = torch.randn(n, 16, generator=g, device="cuda", dtype=torch.float64)
    AX = A @ X
    assert _probe_rel(AX - U @ (R @ (V.t() @ X)), AX) <= 1e-12
    assert (torch.linalg.norm(U.t() @ (U @ X) - X) / math.sqrt(16)).item() <= 1e-12 * math.sqrt(n)
    assert (torch.linalg.norm(V.t() @ (V @ X) - X) / math.sqrt(16)).item() <= 1e-12 * math.sqrt(n)
