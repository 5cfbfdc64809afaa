"""GPU parity of the FP64-emulation mode (PURL_MODE_FP64_EMU) against the FP64 oracle.

The mode runs the FP64 path's algorithm with every product on the BF16 tensor
cores: 8 fixed-point slices per operand (each operand row carried to 2^-63
of its scale), exact class sums drained into 64-bit integers.  Per term of a
product the slicing (2^-62 of each row or column maximum) and the dropped
slice pairs (s + t >= 8, at most 7 * 2^-64 of 2^e_row 2^e_col <= 28 * 2^-64
of the maxima) stay below 2^-59 (row max)(column max).  The mode is therefore
held to the FP64 path's bars: products within 4 k eps of the row and column scales,
factorizations within 1e-12 (invariants) and 1e-10 (oracle parity on the
determined prefix), the same thresholds as the native FP64 tests.
"""
import numpy as np
import pytest

import oracle
from paper_1812_06007_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


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


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (67, 45, 33), (130, 3, 257), (3, 200, 70), (256, 256, 640),
                                   (129, 97, 1300)])
def test_emu_gemm_matches_oracle(B, ta, tb, m, n, k):
    # rows of op(A) and columns of op(B) with magnitudes spread over 2^+-30:
    # the bound is per entry, relative to that row's and column's scale
    rng = np.random.default_rng(m * 7 + n * 13 + k)
    ra = 2.0 ** rng.integers(-30, 31, size=m)
    cb = 2.0 ** rng.integers(-30, 31, size=n)
    opA = rng.standard_normal((m, k)) * ra[:, None]
    opB = rng.standard_normal((k, n)) * cb[None, :]
    A = opA if ta == "N" else opA.T.copy()
    Bm = opB if tb == "N" else opB.T.copy()
    C0 = rng.standard_normal((m, n))
    got = _host(B.purl_gemm_tc(ta, tb, _dev(A), _dev(Bm), alpha=-0.75, beta=0.5, C=_dev(C0), slices=8, exact=True))
    ref = oracle.gemm(ta, tb, A, Bm, alpha=-0.75, beta=0.5, C=C0)
    scale = np.abs(opA).max(axis=1)[:, None] * np.abs(opB).max(axis=0)[None, :] * k + np.abs(C0)
    assert np.all(np.abs(got - ref) <= 4 * k * EPS * scale)


def test_emu_gemm_beats_four_slices(B):
    # the 8-slice configuration is FP64-accurate where 4 slices stop at 2^-32
    rng = np.random.default_rng(5)
    m, n, k = 256, 192, 4096
    A = rng.standard_normal((m, k))
    Bm = rng.standard_normal((k, n))
    ref = A @ Bm
    scale = np.abs(ref).max()
    e7 = np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=8, exact=True)) - ref).max() / scale
    e4 = np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=4, exact=True)) - ref).max() / scale
    assert e7 < 1e-14, e7
    assert e4 > 100 * e7


def test_emu_gemm_cancellation_is_exact(B):
    # A B with exactly cancelling terms: integers below 2^26 (4 of the 8 digits
    # carry them exactly), the second half of each row of A the negated first
    # half and B's two row halves equal, so every entry is exactly 0 while the
    # partial sums reach 2^61 -- beyond FP64's 53 bits, so only exact sums
    # across the 128-deep chunks give 0
    rng = np.random.default_rng(8)
    m, k = 130, 2 * 700
    A = rng.integers(-2**26, 2**26, size=(m, k)).astype(np.float64)
    half = rng.integers(-2**26, 2**26, size=(k // 2, 64)).astype(np.float64)
    Bm = np.vstack([half, half])
    A[:, k // 2:] = -A[:, :k // 2]
    got = _host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=8, exact=True))
    assert np.array_equal(got, np.zeros((m, 64)))


def _determined_prefix(A, q, reorth, tol=1e-12, delta=1e-15):
    n = A.shape[1]
    G = oracle.gaussian(W.SEED_G, n, n)
    Gp = G * (1.0 + delta * np.random.default_rng(99).standard_normal(G.shape))
    U0, R0, V0 = oracle.urv_g(A, G, q, reorth)
    U1, R1, V1 = oracle.urv_g(A, Gp, q, reorth)
    d0, d1 = np.abs(np.diag(R0)), np.abs(np.diag(R1))
    ok = (np.abs(d0 - d1) <= tol * d0) \
        & (np.abs(V0 - V1).max(axis=0) <= tol) & (np.abs(U0 - U1).max(axis=0) <= tol)
    J = int(np.argmin(ok)) if not ok.all() else n
    return J, (U0, R0, V0)


def _check_urv(A, U, R, V, Uo, Ro, Vo, J, tol_inv=1e-12, tol_par=1e-10):
    n = A.shape[1]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ R @ V.T) <= tol_inv * nA
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= tol_inv
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= tol_inv
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert np.all(np.diag(R) >= 0)
    d, do = np.diag(R)[:J], np.diag(Ro)[:J]
    assert np.all(np.abs(d - do) <= tol_par * do)
    assert np.abs(V[:, :J] - Vo[:, :J]).max(initial=0) <= tol_par
    assert np.abs(U[:, :J] - Uo[:, :J]).max(initial=0) <= tol_par


@pytest.mark.parametrize("m,n,q,reorth,profile", [
    (512, 512, 2, True, "exponential"),
    (700, 600, 2, True, "exponential"),
    (300, 200, 1, True, "polynomial"),
    (300, 200, 3, True, "step"),
    (129, 65, 0, True, "exponential"),
    (97, 97, 2, False, "polynomial"),
    (64, 1, 2, True, "exponential"),
    (1, 1, 1, True, "exponential"),
])
def test_emu_urv_matches_oracle(B, m, n, q, reorth, profile):
    A = W.test_matrix_np(m, n, W.sigma_profile(profile, n, decades=8))
    J, (Uo, Ro, Vo) = _determined_prefix(A, q, reorth)
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), q, reorth, W.SEED_G, mode=B.PURL_MODE_FP64_EMU))
    _check_urv(A, U, R, V, Uo, Ro, Vo, J)
    assert B.purl_device_status() == B.PURL_OK


def test_emu_urv_gaussian_entry_matrix_and_fp64_agreement(B):
    A = W.gaussian_matrix_np(1100, 640, 5)
    J, (Uo, Ro, Vo) = _determined_prefix(A, 2, True)
    assert J >= 320
    Ue, Re, Ve = (_host(x) for x in B.purl_urv_factor(_dev(A), 2, True, W.SEED_G, mode=B.PURL_MODE_FP64_EMU))
    _check_urv(A, Ue, Re, Ve, Uo, Ro, Vo, J)
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), 2, True, W.SEED_G))
    assert np.abs(Re - R).max() <= 1e-11 * np.abs(R).max()
    assert np.abs(Ve - V).max() <= 1e-11


@pytest.mark.parametrize("m,n", [(1, 1), (33, 33), (130, 96), (700, 600), (1500, 520)])
def test_emu_qr_matches_oracle(B, m, n):
    M = np.random.default_rng(m + 31 * n).standard_normal((m, n))
    Q, R = B.purl_qr(_dev(M), mode=B.PURL_MODE_FP64_EMU)
    Q, R = _host(Q), _host(R)
    Qo, Ro = oracle.qr(M)
    assert np.abs(Q - Qo).max() < 1e-12
    assert np.abs(R - Ro).max() < 1e-12 * np.abs(Ro).max()
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert np.all(np.diag(R) >= 0)


def test_emu_ulv_of_wide_matrix(B):
    m, n = 200, 330
    A = np.asfortranarray(W.test_matrix_np(n, m, np.linspace(1.0, 0.5, m), seed_u=45, seed_v=46).T)
    U, L, V = (_host(x) for x in B.purl_ulv_factor_ex(_dev(A), 2, True, W.SEED_G, mode=B.PURL_MODE_FP64_EMU))
    Uo, Lo, Vo = oracle.ulv(A, 2, True, W.SEED_G)
    assert np.linalg.norm(A - U @ L @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)
    for X, Xo in ((U, Uo), (L, Lo), (V, Vo)):
        assert np.abs(X - Xo).max() <= 1e-10 * max(1.0, np.abs(Xo).max())
