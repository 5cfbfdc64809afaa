"""Pins for the FP64 oracle, against things other than the oracle itself.

Each test fixes the oracle to something the paper or the mathematics fixes:
an independent library run (numpy's Philox, LAPACK QR/SVD, numpy matmul),
a closed form, an exact invariant of any URV factorization (Section 1), the
Lemma of Section 6, or a special case with a known answer.  A plausible slip
in the oracle (a dropped or transposed power-step product, a wrong sign
convention, a misplaced re-orthonormalisation, an off-by-one in truncation)
makes at least one of them fail.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_06007_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def _numpy_philox_block(ctr0: int, key):
    """Block `ctr0` of numpy's independent Philox4x64-10 (numpy bumps the counter
    before producing a block, so start it one below)."""
    start = (ctr0 - 1) % (1 << 64)
    c = [start, 0, 0, 0] if ctr0 != 0 else [(1 << 64) - 1] * 4
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr0", [0, 1, 2, 3, 17, 1 << 33, (1 << 64) - 2])
@pytest.mark.parametrize("key", [(0, 0), (7, 0), (7, 3), (0xDEADBEEFCAFEF00D, 0x0123456789ABCDEF)])
def test_philox_matches_numpy(ctr0, key):
    mine = oracle.philox4x64_10([ctr0, 0, 0, 0], key)
    assert np.array_equal(mine, _numpy_philox_block(ctr0, key))


def test_uniform_stream_layout():
    # element e is word e%4 of block e/4, top 53 bits centred in their cell
    u = oracle.uniforms(7, 23)
    for e in range(23):
        w = int(_numpy_philox_block(e // 4, (7, 0))[e % 4])
        assert u[e] == ((w >> 11) + 0.5) * 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def test_gaussian_distribution():
    from scipy import stats
    G = oracle.gaussian(123, 1000, 1000)
    z = G.ravel(order="F")
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # pairs from one Box-Muller draw are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5 / math.sqrt(n / 2)


def test_gaussian_layout_is_column_major_linear_index():
    G = oracle.gaussian(5, 7, 3)
    flat = oracle.gaussian(5, 21, 1)[:, 0]
    assert np.array_equal(G.ravel(order="F"), flat)
    assert not np.array_equal(oracle.gaussian(5, 7, 3, stream=1), G)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_gemm_vs_numpy(ta, tb):
    rng = np.random.default_rng(3)
    m, n, k = 13, 7, 11
    A = rng.standard_normal((m, k) if ta == "N" else (k, m))
    B = rng.standard_normal((k, n) if tb == "N" else (n, k))
    C0 = rng.standard_normal((m, n))
    ref = 0.5 * (A if ta == "N" else A.T) @ (B if tb == "N" else B.T) - 2.0 * C0
    got = oracle.gemm(ta, tb, A, B, alpha=0.5, beta=-2.0, C=C0)
    assert np.allclose(got, ref, rtol=0, atol=1e-13)


# ------------------------------------------------------------------ QR ----
def _np_qr_signfixed(M):
    Q, R = np.linalg.qr(M)
    d = np.sign(np.diag(R))
    d[d == 0] = 1
    return Q * d, (R.T * d).T


@pytest.mark.parametrize("m,n", [(1, 1), (5, 5), (40, 40), (60, 40), (129, 65)])
def test_qr_matches_lapack_after_sign_fix(m, n):
    M = np.random.default_rng(m * 1000 + n).standard_normal((m, n))
    Q, R = oracle.qr(M)
    Qn, Rn = _np_qr_signfixed(M)
    assert np.abs(Q - Qn).max() < 1e-13
    assert np.abs(R - Rn).max() < 1e-13 * max(1, np.abs(M).max() * n)
    assert np.all(np.diag(R) >= 0)
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R))


def test_qr_of_orthogonal_is_identity():
    Q0 = W.haar_np(50, 50, 11)
    Q, R = oracle.qr(Q0)
    assert np.abs(R - np.eye(50)).max() < 1e-14 * 50
    assert np.abs(Q - Q0).max() < 1e-14 * 50
    Q, R = oracle.qr(3.5 * Q0)
    assert np.abs(R - 3.5 * np.eye(50)).max() < 1e-13 * 50


def test_qr_of_upper_triangular_positive_diag():
    rng = np.random.default_rng(1)
    T = np.triu(rng.standard_normal((30, 30)))
    T[np.diag_indices(30)] = np.abs(T[np.diag_indices(30)]) + 1.0
    Q, R = oracle.qr(T)
    assert np.array_equal(Q, np.eye(30))  # every reflector is the identity (tau = 0)
    assert np.array_equal(R, T)


def test_qr_sign_convention_on_negative_identity():
    Q, R = oracle.qr(-np.eye(6))
    assert np.array_equal(R, np.eye(6))
    assert np.array_equal(Q, -np.eye(6))


def test_qr_rank_deficient_column():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((20, 8))
    M[:, 3] = 0.0
    M[:, 5] = M[:, 1] * 2.0
    Q, R = oracle.qr(M)
    assert np.abs(Q @ R - M).max() < 1e-13
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-13
    assert np.all(np.diag(R) >= 0) and abs(R[3, 3]) < 1e-14


def test_householder_reflectors_are_lapack_compatible():
    # tau in [1, 2] for nonzero reflectors, v(0) = 1 implicit: H = I - tau v v^T orthogonal
    M = np.random.default_rng(4).standard_normal((12, 5))
    F, tau = oracle.householder_qr(M)
    for j in range(5):
        v = np.zeros(12)
        v[j] = 1.0
        v[j + 1:] = F[j + 1:, j]
        H = np.eye(12) - tau[j] * np.outer(v, v)
        assert np.abs(H @ H.T - np.eye(12)).max() < 1e-14
        assert 1.0 <= tau[j] <= 2.0


# ----------------------------------------------------------------- URV ----
def _invariants(A, U, R, V, tol):
    m, n = A.shape
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A - U @ R @ V.T) <= tol * nA
    assert np.linalg.norm(U.T @ U - np.eye(n)) <= tol
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= tol
    assert np.linalg.norm(V @ V.T - np.eye(n)) <= tol
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert np.all(np.diag(R) >= 0)


@pytest.mark.parametrize("m,n", [(1, 1), (2, 1), (17, 17), (65, 33), (96, 96)])
@pytest.mark.parametrize("q", [0, 1, 2, 3])
@pytest.mark.parametrize("reorth", [False, True])
def test_urv_is_a_urv_factorization(m, n, q, reorth):
    A = W.test_matrix_np(m, n, W.sigma_profile("exponential", n, decades=6))
    U, R, V = oracle.urv(A, q, reorth, W.SEED_G)
    _invariants(A, U, R, V, 20 * max(m, n) * EPS)


def test_urv_frobenius_and_determinant():
    n = 64
    sig = W.sigma_profile("polynomial", n, power=1.0)
    A = W.test_matrix_np(n, n, sig)
    U, R, V = oracle.urv(A, 2, True, W.SEED_G)
    # U, V orthogonal => ||R||_F = ||A||_F and prod |R_jj| = |det A| = prod sigma_j
    assert abs(np.linalg.norm(R) - np.linalg.norm(sig)) < 1e-13 * np.linalg.norm(sig)
    assert abs(np.sum(np.log(np.diag(R))) - np.sum(np.log(sig))) < 1e-10


def test_q0_is_ddh_urv():
    # q = 0: V is the orthonormal factor of G (Section 3: "when q = 0, is DDH-URV")
    n = 40
    A = W.test_matrix_np(50, n, W.sigma_profile("exponential", n, decades=4))
    U, R, V = oracle.urv(A, 0, True, W.SEED_G)
    G = oracle.gaussian(W.SEED_G, n, n)
    Vg, _ = _np_qr_signfixed(G)
    assert np.abs(V - Vg).max() < 1e-13
    Ur, Rr = _np_qr_signfixed(A @ Vg)
    assert np.abs(U - Ur).max() < 1e-12 and np.abs(R - Rr).max() < 1e-13


def _projector(X):
    Q, _ = np.linalg.qr(X)
    return Q @ Q.T


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("ell", [1, 5, 20])
def test_lemma_range_of_leading_U_columns(q, ell):
    # Section 6, Lemma: U(:,1:l) U(:,1:l)^T A = U_rsvd U_rsvd^T A, with the RSVD
    # started from G(:,1:l); its proof shows both bases span A (A^T A)^q G(:,1:l)
    # (Eq. 11) and that V(:,1:l) spans (A^T A)^q G(:,1:l).
    m, n = 70, 50
    A = W.test_matrix_np(m, n, W.sigma_profile("exponential", n, decades=2))
    U, R, V = oracle.urv(A, q, False, W.SEED_G)
    G = oracle.gaussian(W.SEED_G, n, n)[:, :ell]
    Y = G
    for _ in range(q):
        Y = A.T @ (A @ Y)
    Qr = np.linalg.qr(A @ Y)[0]
    P_U = U[:, :ell] @ U[:, :ell].T
    assert np.linalg.norm(P_U @ A - Qr @ (Qr.T @ A), 2) < 1e-10 * np.linalg.norm(A, 2)
    assert np.linalg.norm(P_U - _projector(A @ Y), 2) < 1e-10
    assert np.linalg.norm(V[:, :ell] @ V[:, :ell].T - _projector(Y), 2) < 1e-10


def test_reorthonormalisation_leaves_V_unchanged_in_exact_arithmetic():
    # Q(A Y) = A Y R^-1 with R upper triangular, diag > 0, and Q(M R^-1) = Q(M):
    # with the nonnegative-diagonal convention the re-orthonormalised and plain
    # power iterations give the same V (differences are rounding only).
    m, n = 60, 40
    A = W.test_matrix_np(m, n, W.sigma_profile("exponential", n, decades=1))
    for q in (1, 2, 3):
        _, _, V0 = oracle.urv(A, q, False, W.SEED_G)
        _, _, V1 = oracle.urv(A, q, True, W.SEED_G)
        assert np.abs(V0 - V1).max() < 1e-9


def test_transposed_power_step_would_be_caught():
    # the Lemma test above distinguishes A^T A from A A^T: for a non-symmetric
    # square A the two Krylov ranges differ, so guard that the check has teeth.
    n = 30
    A = W.test_matrix_np(n, n, W.sigma_profile("exponential", n, decades=1))
    G = oracle.gaussian(W.SEED_G, n, n)[:, :5]
    assert np.linalg.norm(_projector(A.T @ A @ G) - _projector(A @ A.T @ G), 2) > 1e-3


def test_orthogonal_and_scaled_identity_inputs():
    n = 32
    Q0 = W.haar_np(n, n, 21)
    U, R, V = oracle.urv(Q0, 2, True, W.SEED_G)
    assert np.abs(R - np.eye(n)).max() < 1e-13
    assert np.abs(U - Q0 @ V).max() < 1e-13
    U, R, V = oracle.urv(2.5 * np.eye(n), 1, True, W.SEED_G)
    assert np.abs(R - 2.5 * np.eye(n)).max() < 1e-13
    assert np.abs(U - V).max() < 1e-13


def test_rank_one_input():
    m, n = 40, 25
    rng = np.random.default_rng(8)
    u = rng.standard_normal(m); u /= np.linalg.norm(u)
    v = rng.standard_normal(n); v /= np.linalg.norm(v)
    A = 3.0 * np.outer(u, v)
    U, R, V = oracle.urv(A, 1, True, W.SEED_G)
    assert abs(R[0, 0] - 3.0) < 1e-13
    assert abs(abs(V[:, 0] @ v) - 1.0) < 1e-13
    assert np.abs(np.diag(R)[1:]).max() < 1e-13
    assert np.linalg.norm(A - U @ R @ V.T) < 1e-13


def test_rank_revealing_interlacing_holds_for_every_k():
    # For any URV, R has A's singular values, so sigma_min(R11) <= sigma_k(A) and
    # ||R22||_2 >= sigma_{k+1}(A) (Section 1, Eq. 2 partition).
    m, n = 45, 30
    A = W.test_matrix_np(m, n, W.sigma_profile("polynomial", n, power=1.0))
    s = np.linalg.svd(A, compute_uv=False)
    for q in (0, 1, 2):
        _, R, _ = oracle.urv(A, q, True, W.SEED_G)
        for k in range(1, n):
            r11 = np.linalg.svd(R[:k, :k], compute_uv=False)
            r22 = np.linalg.svd(R[k:, k:], compute_uv=False)
            assert r11[-1] <= s[k - 1] * (1 + 1e-12)
            assert r22[0] >= s[k] * (1 - 1e-12)


def test_power_steps_sharpen_rank_revealing_diagonal():
    # Section 3 / Fig. 3: with q >= 1, |R_jj| tracks sigma_j far better than q = 0.
    n = 120
    sig = W.sigma_profile("exponential", n, decades=10)
    A = W.test_matrix_np(150, n, sig)
    dev = []
    for q in (0, 1, 2):
        _, R, _ = oracle.urv(A, q, True, W.SEED_G)
        d = np.abs(np.diag(R))
        dev.append(np.median(np.abs(np.log10(d[: n // 2] / sig[: n // 2]))))
    assert dev[1] < dev[0] and dev[2] <= dev[1] * 1.05
    assert dev[2] < 0.25


# ------------------------------------------------------ truncation / SVD ----
def test_jacobi_svd_vs_lapack_and_closed_form():
    d = np.array([5.0, 3.0, 2.0, 1e-3, 0.0])
    assert np.allclose(oracle.jacobi_svd(np.diag(d)), d, rtol=0, atol=1e-15)
    A = np.random.default_rng(5).standard_normal((32, 24))
    assert np.allclose(oracle.jacobi_svd(A), np.linalg.svd(A, compute_uv=False), rtol=1e-12, atol=0)


def test_truncation_definitions_and_eckart_young():
    m, n = 32, 24
    A = W.test_matrix_np(m, n, W.sigma_profile("exponential", n, decades=5))
    U, R, V = oracle.urv(A, 1, True, W.SEED_G)
    s = oracle.jacobi_svd(A)
    assert np.abs(oracle.truncate(U, R, V, n) - A).max() < 1e-14
    assert np.abs(oracle.truncate(U, R, V, 0)).max() == 0.0
    for k in range(1, n):
        Ak = oracle.truncate(U, R, V, k)
        # A_k = U_k U_k^T A (U_k^T A = R(1:k,:) V^T) and rank k
        assert np.abs(Ak - U[:, :k] @ (U[:, :k].T @ A)).max() < 1e-13
        assert np.linalg.matrix_rank(Ak, tol=1e-10 * s[0]) <= k
        err2 = np.linalg.svd(A - Ak, compute_uv=False)[0]
        assert err2 >= s[k] * (1 - 1e-10)


def test_urv_rejects_wide_matrix():
    with pytest.raises(ValueError):
        oracle.urv(np.zeros((3, 5)), 1, True, 1)


def test_golden_fixture_reproduces(tmp_path):
    # tests/golden/urv_64x48_q2.txt was written by tests/golden/make_golden.py
    # (oracle only) on x86-64; the oracle must reproduce it on any host.
    import os
    from tests.golden.make_golden import CASES, compute_case, load_fixture
    here = os.path.join(os.path.dirname(__file__), "golden")
    for name in CASES:
        got = compute_case(name)
        ref = load_fixture(os.path.join(here, name + ".txt"))
        for key in ref:
            assert np.allclose(got[key], ref[key], rtol=1e-12, atol=1e-14), (name, key)


# ------------------------------------------------------------ ULV (m < n) --
@pytest.mark.parametrize("m,n,q,reorth", [(7, 12, 1, True), (20, 31, 2, True), (16, 16, 0, True), (9, 30, 2, False)])
def test_ulv_invariants(m, n, q, reorth):
    # Section 1: the wide case through A^T.  Pinned by what a ULV must satisfy,
    # not by re-deriving it: A = U L V^T, L lower triangular with diag >= 0,
    # orthonormal U and V, ||L||_F = ||A||_F, and the interlacing bounds of a
    # triangular factor against the singular values of A (numpy's SVD).
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n))
    U, L, V = oracle.ulv(A, q, reorth, 7)
    assert U.shape == (m, m) and L.shape == (m, m) and V.shape == (n, m)
    eps = np.finfo(float).eps
    assert np.linalg.norm(A - U @ L @ V.T) <= 50 * n * eps * np.linalg.norm(A)
    assert np.linalg.norm(np.eye(m) - U.T @ U) <= 50 * n * eps
    assert np.linalg.norm(np.eye(m) - V.T @ V) <= 50 * n * eps
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)
    assert abs(np.linalg.norm(L) - np.linalg.norm(A)) <= 1e-12 * np.linalg.norm(A)
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(1, m):
        assert np.linalg.svd(L[:k, :k], compute_uv=False)[-1] <= s[k - 1] * (1 + 1e-12)
        assert np.linalg.norm(L[k:, k:], 2) >= s[k] * (1 - 1e-12)


def test_ulv_rejects_tall():
    with pytest.raises(ValueError):
        oracle.ulv(np.zeros((5, 3)), 1, True, 7)
