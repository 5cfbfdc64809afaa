"""FP32 precision on the tensor cores (PURL_MODE_FP32), the FP32-storage entry
points, and the reverse mode run on the tensor cores (purl_urv_backward_ex in
PURL_MODE_FP64_EMU and PURL_MODE_FP32), against the FP64 oracle.

Bars.  FP32 mode: every product carries each operand row to 2^-32 of its
scale (4 exact slices), so entries down to 2^-8 of their row's maximum keep
FP32's unit roundoff u = 2^-24; the factorization is held to FP32 Householder
bounds of the gamma_{4n} = 4 n u form: relative reconstruction and
||I - Q^T Q||_F at most 4 n u, and |R(j,j)| within a median 1e-3 of the
oracle where sigma_j / sigma_1 >= 1e-2 (its absolute error is about
sqrt(n) u sigma_1, i.e. ~1e-4 of sigma_j there).  FP64-emulated backward: the
FP64 path's bars (1e-10 of the largest entry against the oracle's reverse
mode; 1e-8 in the Frobenius norm against the projection formula at 2048).
FP32 backward: the error of the inputs to the R^{-T} solves (~sqrt(n) u) is
amplified by cond(R): 2e-4 of the largest entry for the cond <= 3.3
matrices, 5e-2 in the Frobenius norm at 2048 (Gaussian A, cond ~ 1e4:
45 * 6e-8 * 1e4 ~ 3e-2).
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as oadj
from paper_1812_06007_gb300 import workloads as W
from tests.test_gpu_fp64 import _check_urv, _determined_prefix

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _dev(x, dtype=None):
    import torch
    from paper_1812_06007_gb300.binding import as_colmajor
    t = as_colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())
    return t if dtype is None else t.to(dtype).t().contiguous().t()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def _wellcond(m, n, seed, lo=0.3):
    return W.test_matrix_np(m, n, np.linspace(1.0, lo, n), seed_u=seed, seed_v=seed + 1)


def _cotangents(m, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((m, n)), rng.standard_normal((n, n)), rng.standard_normal((n, n)))


@pytest.mark.parametrize("m,n,q,reorth,profile", [
    (512, 512, 2, True, "exponential"),
    (300, 200, 1, True, "polynomial"),
    (257, 129, 0, True, "exponential"),
    (96, 96, 3, True, "step"),
    (600, 520, 2, True, "exponential"),
])
def test_fp32_mode_urv_matches_oracle_at_fp32_bounds(B, m, n, q, reorth, profile):
    sig = W.sigma_profile(profile, n, decades=6)
    A = W.test_matrix_np(m, n, sig)
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), q, reorth, W.SEED_G, mode=B.PURL_MODE_FP32))
    nA = np.linalg.norm(A)
    recon = np.linalg.norm(A - U @ R @ V.T) / nA
    ou, ov = np.linalg.norm(U.T @ U - np.eye(n)), np.linalg.norm(V.T @ V - np.eye(n))
    _, Ro, _ = oracle.urv(A, q, reorth, W.SEED_G)
    lead = sig / sig[0] >= 1e-2
    dev = np.abs(np.diag(R)[lead] - np.diag(Ro)[lead]) / np.diag(Ro)[lead]
    print(f"\nfp32 {m}x{n} q={q} {profile}: recon={recon:.2e} orthU={ou:.2e} orthV={ov:.2e} "
          f"|Rjj| median dev={np.median(dev):.2e} (bound 4nu={4 * n * U32:.2e})")
    assert recon <= 4 * n * U32 and ou <= 4 * n * U32 and ov <= 4 * n * U32
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n))) and np.all(np.diag(R) >= 0)
    assert np.median(dev) <= 1e-3
    assert B.purl_device_status() == B.PURL_OK


def test_fp32_storage_entry_equals_rounded_fp32_mode(B):
    # A given in FP32: the FP32 entry point widens it exactly and runs the same
    # mode, so its outputs are the FP32 roundings of the FP64-interface call
    import torch
    m, n = 300, 240
    A = W.test_matrix_np(m, n, W.sigma_profile("exponential", n, decades=5)).astype(np.float32).astype(np.float64)
    U32_, R32_, V32_ = B.purl_urv_factor_f32(_dev(A, torch.float32), 2, True, W.SEED_G)
    U, R, V = B.purl_urv_factor(_dev(A), 2, True, W.SEED_G, mode=B.PURL_MODE_FP32)
    for got, ref in ((U32_, U), (R32_, R), (V32_, V)):
        assert got.dtype == torch.float32
        assert np.array_equal(_host(got), _host(ref.to(torch.float32)))
    # other modes through the FP32 entry point
    Ue, Re, Ve = B.purl_urv_factor_f32(_dev(A, torch.float32), 2, True, W.SEED_G, mode=B.PURL_MODE_FP64_EMU)
    Uo, Ro, Vo = oracle.urv(A, 2, True, W.SEED_G)
    assert np.abs(_host(Re) - Ro).max() <= 2 * U32 * np.abs(Ro).max()


@pytest.mark.parametrize("m,n,q,reorth", [(64, 64, 2, True), (200, 136, 1, True), (256, 256, 2, False),
                                          (130, 33, 3, True)])
def test_emulated_backward_matches_oracle(B, m, n, q, reorth):
    A = _wellcond(m, n, 500 + m + n)
    # the forward pass it differentiates is the FP64-emulation forward
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), q, reorth, W.SEED_G, mode=B.PURL_MODE_FP64_EMU))
    Uo, Ro, Vo = oracle.urv(A, q, reorth, W.SEED_G)
    assert np.abs(R - Ro).max() <= 1e-12 * np.abs(Ro).max()
    Ub, Rb, Vb = _cotangents(m, n, 3 + q)
    got = _host(B.purl_urv_backward_ex(_dev(A), q, reorth, W.SEED_G, _dev(Ub), _dev(Rb), _dev(Vb),
                                       mode=B.PURL_MODE_FP64_EMU))
    ref = oadj.urv_backward(A, q, reorth, W.SEED_G, Ub, Rb, Vb)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), np.abs(got - ref).max()


@pytest.mark.parametrize("m,n,q,reorth", [(64, 64, 2, True), (200, 136, 1, True), (300, 256, 2, True)])
def test_fp32_backward_matches_oracle(B, m, n, q, reorth):
    import torch
    A = _wellcond(m, n, 500 + m + n).astype(np.float32).astype(np.float64)
    Ub, Rb, Vb = (x.astype(np.float32).astype(np.float64) for x in _cotangents(m, n, 3 + q))
    ref = oadj.urv_backward(A, q, reorth, W.SEED_G, Ub, Rb, Vb)
    got = _host(B.purl_urv_backward_ex(_dev(A), q, reorth, W.SEED_G, _dev(Ub), _dev(Rb), _dev(Vb),
                                       mode=B.PURL_MODE_FP32))
    err = np.abs(got - ref).max() / np.abs(ref).max()
    got32 = _host(B.purl_urv_backward_f32(*(_dev(x, torch.float32) for x in (A,)), q, reorth, W.SEED_G,
                                          *(_dev(x, torch.float32) for x in (Ub, Rb, Vb))))
    print(f"\nfp32 backward {m}x{n} q={q}: max rel err {err:.2e}")
    assert err <= 2e-4
    # the FP32 entry point is the FP64-interface FP32 mode rounded once
    assert np.array_equal(got32, got.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("mode", ["fp32", "emu"])
def test_adjoint_2048_tensor_core_modes_match_projection_formula(B, mode):
    # configuration of the adjoint workload: m = n = 2048, q = 2, reorth, k = 512,
    # Gaussian A, B ~ N(0,1); FP32 mode on FP32 tensors, FP64 emulation on FP64
    import torch
    from paper_1812_06007_gb300 import autograd
    m = n = 2048
    k, q = 512, 2
    A = W.gaussian_matrix_np(m, n, 2048)
    Bt = np.random.default_rng(W.SEED_B).standard_normal((m, n))
    if mode == "fp32":
        A = A.astype(np.float32).astype(np.float64)
        Bt = Bt.astype(np.float32).astype(np.float64)
        At = _dev(A, torch.float32).requires_grad_(True)
        L = autograd.truncated_loss(At, q, True, W.SEED_G, k, _dev(Bt, torch.float32))
        bar_l, bar_g = 1e-5, 5e-2
    else:
        At = _dev(A).requires_grad_(True)
        L = autograd.truncated_loss(At, q, True, W.SEED_G, k, _dev(Bt), mode=B.PURL_MODE_FP64_EMU)
        bar_l, bar_g = 1e-9, 1e-8
    L.backward()
    got = _host(At.grad)
    G = oracle.gaussian(W.SEED_G, n, n)
    Lo, ref = oadj.truncated_loss_grad_projection(A, G, q, k, Bt)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\nadjoint 2048 {mode}: loss rel {abs(float(L.detach()) - Lo) / Lo:.2e}, gradient rel {rel:.2e}")
    assert abs(float(L.detach()) - Lo) <= bar_l * Lo
    assert rel <= bar_g


def test_mode_arguments(B):
    import ctypes
    L = B.lib()
    nul = ctypes.c_void_p(0)
    assert L.purl_urv_backward_ex_workspace_bytes(64, 64, 2, B.PURL_MODE_MIXED_BF16) == 0
    assert L.purl_urv_backward_ex_workspace_bytes(64, 64, 2, B.PURL_MODE_FP32) > 0
    assert L.purl_urv_f32_workspace_bytes(64, 64, 99) == 0
    fake = ctypes.c_void_p(256)
    assert L.purl_urv_backward_ex(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, 4, fake, 4, 2, nul, 0, nul) == -16
    assert L.purl_urv_factor_f32(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, 4, 99, nul, 0, nul) == -14
