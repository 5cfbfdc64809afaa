"""GPU randomized SVD (purl_rsvd, Section 6) against the oracle's RSVD (same
G prefix, same sign convention) and against the paper's Lemma on the GPU's own
PowerURV.  FP64: singular values to 1e-12 of S_0 plus the rounding of the
power iteration amplified by (S_0/S_{l-1})^p (p = 1 re-orthonormalised,
2q + 1 plain); U, V to 1e-9 on directions resolved to 1e-11 and separated by
>= 5% from their neighbours (vector error ~ u/gap); Lemma:
||P_U_rsvd - P_U(:,1:l)||_2 <= 1e-9."""
import numpy as np
import pytest

from oracle import rsvd as orsvd
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


@pytest.mark.parametrize("m,n,l,q,reorth", [(300, 200, 60, 1, False), (300, 200, 60, 2, True), (129, 129, 33, 0, False),
                                            (500, 260, 100, 2, True), (70, 64, 1, 1, True), (256, 256, 255, 1, True)])
def test_rsvd_matches_oracle(B, m, n, l, q, reorth):
    sig = 0.9 ** np.arange(n)  # 10% gaps
    A = W.test_matrix_np(m, n, sig, seed_u=50 + l, seed_v=51 + l)
    U, S, V = (_host(t) for t in B.purl_rsvd(_dev(A), l, q, W.SEED_G, reorth))
    Uo, So, Vo = orsvd.rsvd(A, l, q, W.SEED_G, reorth)
    # rounding reaches direction j of the range amplified by (S_0/S_j)^p: p = 1
    # when every product works on orthonormal iterates, p = 2q + 1 for the plain
    # power iteration (Y = A (A^T A)^q G is rounded against S_0^(2q+1))
    eps = np.finfo(float).eps
    p = 1 if (reorth or q == 0) else 2 * q + 1
    amp = eps * (So[0] / np.maximum(So, 1e-300)) ** p
    assert np.all(np.abs(S - So) <= 1e-12 * So[0] + 10 * amp[-1] * So[0])
    assert np.all(np.diff(S) <= 0)
    # vectors: resolved directions (amp <= 1e-11) with a gap >= 5% to both neighbours
    gaps = np.minimum(np.abs(np.diff(So, prepend=np.inf)), np.abs(np.diff(So, append=-np.inf))) / So
    ok = (gaps >= 0.05) & (amp <= 1e-11)
    if l < n:
        ok[-1] = False  # the last kept direction feels the truncation most
    assert ok[: min(l, 8)].all() or l < 8
    assert np.abs(U[:, ok] - Uo[:, ok]).max(initial=0.0) <= 1e-9
    assert np.abs(V[:, ok] - Vo[:, ok]).max(initial=0.0) <= 1e-9
    assert np.linalg.norm(U.T @ U - np.eye(l)) <= 1e-12 * l
    assert np.linalg.norm(V.T @ V - np.eye(l)) <= 1e-12 * l


def test_rsvd_exact_rank_recovers_matrix(B):
    m, n, r, l = 400, 300, 20, 24
    sig = np.zeros(n)
    sig[:r] = np.linspace(2.0, 1.0, r)
    A = W.test_matrix_np(m, n, sig, seed_u=3, seed_v=4)
    U, S, V = (_host(t) for t in B.purl_rsvd(_dev(A), l, 1, W.SEED_G))
    assert np.linalg.norm(A - (U * S) @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(S[:r], sig[:r], rtol=1e-12, atol=0)


def test_lemma_on_the_gpu(B):
    # range(U_rsvd) == range(U(:, 1:l)) of the library's own PowerURV, same seed
    m, n, l = 400, 300, 40
    A = W.test_matrix_np(m, n, np.linspace(1.0, 0.3, n), seed_u=8, seed_v=9)
    Ur = _host(B.purl_rsvd(_dev(A), l, 2, W.SEED_G, True)[0])
    U = _host(B.purl_urv_factor(_dev(A), 2, True, W.SEED_G)[0])[:, :l]
    assert np.linalg.norm(Ur @ Ur.T - U @ U.T, 2) <= 1e-9
