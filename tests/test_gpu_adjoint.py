"""GPU reverse mode of PowerURV (purl_urv_backward, FP64, G fixed) against the
oracle's reverse mode, FP64 finite differences of the GPU forward pass, the
k = n identity, and the QR-free projection-formula gradient of the truncated
loss L = ||A_k - B||_F^2 (A_k = U(:,1:k) R(1:k,:) V^T) at m = n = 2048, k = 512.

Bars: elementwise agreement with the oracle to 1e-10 relative to the largest
entry (both sides FP64; the gradient's condition is that of the R^{-T}
solves, ~cond(A), kept below 10 here); finite differences to 1e-6 relative
(central differences, h = 1e-6); the 2048 gradient to 1e-8 relative in the
Frobenius norm (Gaussian A, cond(A) ~ 1e4, so the R^{-T} solves lose about
four digits on either side).
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import adjoint as oadj
from paper_1812_06007_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _dev(x):
    import torch
    from paper_1812_06007_gb300.binding import as_colmajor
    return as_colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _wellcond(m, n, seed, lo=0.3):
    return W.test_matrix_np(m, n, np.linspace(1.0, lo, n), seed_u=seed, seed_v=seed + 1)


def _cotangents(m, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((m, n)), rng.standard_normal((n, n)), rng.standard_normal((n, n)))


@pytest.mark.parametrize("m,n,q,reorth", [
    (64, 64, 2, True), (64, 64, 0, True), (97, 97, 1, False), (200, 136, 1, True),
    (300, 256, 2, True), (256, 256, 2, False), (130, 33, 3, True), (1, 1, 1, True),
])
def test_backward_matches_oracle(B, m, n, q, reorth):
    A = _wellcond(m, n, 500 + m + n)
    Ub, Rb, Vb = _cotangents(m, n, 3 + q)
    got = _host(B.purl_urv_backward(_dev(A), q, reorth, W.SEED_G, _dev(Ub), _dev(Rb), _dev(Vb)))
    ref = oadj.urv_backward(A, q, reorth, W.SEED_G, Ub, Rb, Vb)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), np.abs(got - ref).max()


def test_backward_drops_lower_triangle_of_rbar(B):
    m, n = 80, 72
    A = _wellcond(m, n, 9)
    Ub, Rb, Vb = _cotangents(m, n, 1)
    a = _host(B.purl_urv_backward(_dev(A), 1, True, 5, _dev(Ub), _dev(Rb), _dev(Vb)))
    b = _host(B.purl_urv_backward(_dev(A), 1, True, 5, _dev(Ub), _dev(np.triu(Rb)), _dev(Vb)))
    assert np.array_equal(a, b)


def test_backward_matches_gpu_finite_differences(B):
    # FP64 central differences of the GPU forward pass itself at n = 64.
    m = n = 64
    q, reorth, seed = 2, True, W.SEED_G
    A = _wellcond(m, n, 71)
    Ub, Rb, Vb = _cotangents(m, n, 8)
    Rb = np.triu(Rb)

    def f(X):
        U, R, V = (_host(t) for t in B.purl_urv_factor(_dev(X), q, reorth, seed))
        return float(np.sum(Ub * U) + np.sum(Rb * R) + np.sum(Vb * V))

    Abar = _host(B.purl_urv_backward(_dev(A), q, reorth, seed, _dev(Ub), _dev(Rb), _dev(Vb)))
    rng = np.random.default_rng(12)
    h = 1e-6
    for _ in range(4):
        D = rng.standard_normal((m, n))
        fd = (f(A + h * D) - f(A - h * D)) / (2 * h)
        an = float(np.sum(Abar * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("m,n,q", [(300, 300, 2), (257, 190, 1)])
def test_truncated_loss_full_rank_gradient_is_identity_gradient(B, m, n, q):
    import torch
    from paper_1812_06007_gb300 import autograd
    A = _wellcond(m, n, 40 + q)
    Bt = np.random.default_rng(W.SEED_B).standard_normal((m, n))
    At = _dev(A).requires_grad_(True)
    L = autograd.truncated_loss(At, q, True, W.SEED_G, n, _dev(Bt))
    L.backward()
    got = _host(At.grad)
    ref = 2.0 * (A - Bt)
    assert abs(float(L.detach()) - np.sum((A - Bt) ** 2)) <= 1e-10 * np.sum((A - Bt) ** 2)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    del torch


def test_truncated_loss_autograd_matches_oracle_small(B):
    from paper_1812_06007_gb300 import autograd
    m = n = 64
    k, q = 16, 2
    A = W.gaussian_matrix_np(m, n, 4)
    Bt = np.random.default_rng(W.SEED_B).standard_normal((m, n))
    At = _dev(A).requires_grad_(True)
    L = autograd.truncated_loss(At, q, True, W.SEED_G, k, _dev(Bt))
    L.backward()
    got = _host(At.grad)
    G = oracle.gaussian(W.SEED_G, n, n)
    U, R, V = oracle.urv_g(A, G, q, True)
    Lo, Ub, Rb, Vb = oadj.truncated_loss_cotangents(U, R, V, k, Bt)
    ref = oadj.urv_backward_g(A, G, q, True, Ub, Rb, Vb)
    assert abs(float(L.detach()) - Lo) <= 1e-10 * Lo
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_adjoint_2048_matches_projection_formula(B):
    # m = n = 2048, q = 2, reorth, k = 512, Gaussian A, B ~ N(0,1): the
    # gradient through both QRs and every power step, against the QR-free
    # projection formula (appendix Lemma), evaluated by the oracle on the host.
    from paper_1812_06007_gb300 import autograd
    m = n = 2048
    k, q = 512, 2
    A = W.gaussian_matrix_np(m, n, 2048)
    Bt = np.random.default_rng(W.SEED_B).standard_normal((m, n))
    At = _dev(A).requires_grad_(True)
    L = autograd.truncated_loss(At, q, True, W.SEED_G, k, _dev(Bt))
    L.backward()
    got = _host(At.grad)
    G = oracle.gaussian(W.SEED_G, n, n)
    Lo, ref = oadj.truncated_loss_grad_projection(A, G, q, k, Bt)
    assert abs(float(L.detach()) - Lo) <= 1e-9 * Lo
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_backward_workspace_and_empty(B):
    import torch
    L = B.lib()
    assert L.purl_urv_backward_workspace_bytes(3, 5, 1) == 0
    need = B.purl_urv_backward_workspace_bytes(96, 80, 2)
    assert need > 0
    A = _wellcond(96, 80, 2)
    Ub, Rb, Vb = _cotangents(96, 80, 2)
    ws = torch.empty(need // 8 + 1, dtype=torch.float64, device="cuda")
    a = _host(B.purl_urv_backward(_dev(A), 2, True, 3, _dev(Ub), _dev(Rb), _dev(Vb), workspace=ws))
    b = _host(B.purl_urv_backward(_dev(A), 2, True, 3, _dev(Ub), _dev(Rb), _dev(Vb)))
    assert np.array_equal(a, b)
    small = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PurlError):
        B.purl_urv_backward(_dev(A), 2, True, 3, _dev(Ub), _dev(Rb), _dev(Vb), workspace=small)
    nul = ctypes.c_void_p(0)
    assert L.purl_urv_backward(0, 0, nul, 1, 1, 1, 7, nul, 1, nul, 1, nul, 1, nul, 1, nul, 0, nul) == 0
