"""Elementwise oracle parity at the sizes where the GPU path changes code path.

- The Householder panel kernel launches ceil(rows / 64) cooperative blocks,
  capped at the SM count: beyond ~10K rows every block owns a slab of more
  than 64 rows.  Tall-skinny QRs of 20000 x 64 and 40000 x 96 take that path,
  as the n = 16384 factorizations of the benchmark do; at 70000 rows the
  tensor-core QR's panel no longer has room for a second shared copy of the
  rounded vectors and rounds them in place.
- The blocked QRs group 32-column panels into 512-column outer blocks whose
  aggregated reflectors update the rest of the matrix: n = 1536 crosses three
  outer blocks (the smaller parity tests cross at most two).

Bars: the FP64 and FP64-emulation modes are held to the FP64 path's bars
(Q elementwise to 1e-12, R to 1e-12 of its largest entry; URV invariants to
1e-12 and |R(j,j)|, U and V columns to 1e-10 on the determined prefix J*,
Section 3); the mixed mode to its own (reconstruction 1e-6, orthogonality
1e-7 per entry, Gaussian-input factors within 1e-5 of FP64).
"""
import numpy as np
import pytest

import oracle
from paper_1812_06007_gb300 import workloads as W
from tests.test_gpu_fp64 import _check_urv, _determined_prefix

pytestmark = pytest.mark.gpu

MODES = ["fp64", "emu", "mixed"]


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _mode(B, name):
    return {"fp64": B.PURL_MODE_FP64, "mixed": B.PURL_MODE_MIXED_BF16, "emu": B.PURL_MODE_FP64_EMU}[name]


def _dev(x):
    import torch
    from paper_1812_06007_gb300.binding import as_colmajor
    return as_colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _check_qr(mode, M, Q, R):
    m, n = M.shape
    Qo, Ro = oracle.qr(M)
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert np.all(np.diag(R) >= 0)
    if mode == "mixed":
        E = Q.T @ Q - np.eye(n)
        assert np.linalg.norm(Q @ R - M) <= 1e-6 * np.linalg.norm(M)
        assert np.abs(E).max() <= 1e-7
        assert np.abs(Q - Qo).max() < 1e-5
        assert np.abs(R - Ro).max() < 1e-5 * np.abs(Ro).max()
    else:
        assert np.abs(Q - Qo).max() < 1e-12
        assert np.abs(R - Ro).max() < 1e-12 * np.abs(Ro).max()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,n", [(20000, 64), (40000, 96), (10241, 33), (70000, 40)])
def test_tall_skinny_qr_on_capped_panel_grid(B, mode, m, n):
    M = np.random.default_rng(m + n).standard_normal((m, n))
    Q, R = (_host(x) for x in B.purl_qr(_dev(M), mode=_mode(B, mode)))
    _check_qr(mode, M, Q, R)
    assert B.purl_device_status() == B.PURL_OK


@pytest.mark.parametrize("mode", MODES)
def test_qr_across_three_outer_blocks(B, mode):
    M = np.random.default_rng(1536).standard_normal((2100, 1536))
    Q, R = (_host(x) for x in B.purl_qr(_dev(M), mode=_mode(B, mode)))
    _check_qr(mode, M, Q, R)


@pytest.mark.parametrize("mode", ["fp64", "emu"])
def test_urv_across_three_outer_blocks_matches_oracle(B, mode):
    n = 1536
    A = W.test_matrix_np(n, n, W.sigma_profile("exponential", n, decades=8))
    J, (Uo, Ro, Vo) = _determined_prefix(A, 2, True)
    assert J >= 64
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), 2, True, W.SEED_G, mode=_mode(B, mode)))
    _check_urv(A, U, R, V, Uo, Ro, Vo, J)
    assert B.purl_device_status() == B.PURL_OK


def test_mixed_urv_across_three_outer_blocks(B):
    # invariants at the mixed bars, and the deviation of the leading, spectrally
    # resolved columns from the FP64 oracle (sigma_j / sigma_1 > 1e-2)
    n = 1536
    sig = W.sigma_profile("exponential", n, decades=6)
    A = W.test_matrix_np(n, n, sig)
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), 2, True, W.SEED_G, mode=B.PURL_MODE_MIXED_BF16))
    Uo, Ro, Vo = oracle.urv(A, 2, True, W.SEED_G)
    nA = np.linalg.norm(A)
    recon = np.linalg.norm(A - U @ R @ V.T) / nA
    eu, ev = U.T @ U - np.eye(n), V.T @ V - np.eye(n)
    assert recon <= 1e-6
    assert np.abs(eu).max() <= 1e-7 and np.abs(ev).max() <= 1e-7
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n))) and np.all(np.diag(R) >= 0)
    lead = sig / sig[0] > 1e-2
    k = int(lead.sum())
    d, do = np.diag(R)[:k], np.diag(Ro)[:k]
    dr = np.abs(d - do) / do
    cu = np.abs(U[:, :k] - Uo[:, :k]).max(axis=0)
    cv = np.abs(V[:, :k] - Vo[:, :k]).max(axis=0)
    print(f"\nmixed urv {n}: recon={recon:.2e} orth_max U={np.abs(eu).max():.2e} V={np.abs(ev).max():.2e}; "
          f"leading {k} columns: |R_jj| rel dev median={np.median(dr):.2e} max={dr.max():.2e}; "
          f"U col max-abs dev median={np.median(cu):.2e} max={cu.max():.2e}; "
          f"V col median={np.median(cv):.2e} max={cv.max():.2e}")
    assert np.median(dr) < 5e-2
