"""Wide matrices (m <= n): purl_ulv_factor_ex, the ULV of A through the URV of
A^T (Section 1), against the oracle's ULV.  FP64: reconstruction and
orthogonality <= 1e-12, U, L, V elementwise to 1e-10 on matrices whose every
column is determined (sigma in [0.5, 1]); mixed: reconstruction <= 1e-6."""
import ctypes

import numpy as np
import pytest

import oracle
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


def _wide(m, n, seed):
    return np.asfortranarray(W.test_matrix_np(n, m, np.linspace(1.0, 0.5, m), seed_u=seed, seed_v=seed + 1).T)


@pytest.mark.parametrize("m,n,q,reorth", [(200, 300, 2, True), (64, 257, 1, True), (96, 96, 0, True),
                                          (130, 400, 2, False), (1, 40, 1, True)])
def test_ulv_fp64_matches_oracle(B, m, n, q, reorth):
    A = _wide(m, n, 40 + m)
    U, L, V = (_host(t) for t in B.purl_ulv_factor_ex(_dev(A), q, reorth, W.SEED_G))
    Uo, Lo, Vo = oracle.ulv(A, q, reorth, W.SEED_G)
    assert np.linalg.norm(A - U @ L @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(np.eye(m) - U.T @ U) <= 1e-12 * np.sqrt(m)
    assert np.linalg.norm(np.eye(m) - V.T @ V) <= 1e-12 * np.sqrt(m)
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)
    for X, Xo in ((U, Uo), (L, Lo), (V, Vo)):
        assert np.abs(X - Xo).max() <= 1e-10 * max(1.0, np.abs(Xo).max())


def test_ulv_mixed_reconstruction(B):
    m, n = 384, 1000
    A = _wide(m, n, 5)
    U, L, V = (_host(t) for t in B.purl_ulv_factor_ex(_dev(A), 2, True, W.SEED_G, mode=B.PURL_MODE_MIXED_BF16))
    assert np.linalg.norm(A - U @ L @ V.T) <= 1e-6 * np.linalg.norm(A)
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)


def test_ulv_argument_errors(B):
    L = B.lib()
    nul = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)
    assert L.purl_ulv_factor_ex(5, 3, fake, 5, 1, 1, 7, fake, 5, fake, 5, fake, 3, 0, nul, 0, nul) == B.PURL_ERR_SHAPE
    assert L.purl_ulv_factor_ex(3, 5, fake, 3, 1, 1, 7, fake, 3, fake, 3, fake, 4, 0, nul, 0, nul) == -13
    assert L.purl_ulv_workspace_bytes(5, 3, 0) == 0
    assert L.purl_ulv_factor_ex(0, 5, nul, 1, 1, 1, 7, nul, 1, nul, 1, nul, 5, 0, nul, 0, nul) == 0
