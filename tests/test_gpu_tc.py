"""GPU parity of the BF16 tensor-core product engine (tcgen05) against the FP64 oracle.

With S slices per operand the representation error of each operand is about
2^(-8S-1) relative and the dropped slice pairs (s + t >= S) about 2^-8S.  The
accumulator is FP32 in tensor memory: every MMA (K = 16) adds into it once, so
a product sees steps = S(S+1)/2 * ceil(k/16) roundings of about 2^-24 of the
running sum; for S = 3 this, not the slicing, is the floor (measured ~8e-7 of
sum |a||b| at k = 64).  The bound checked, element by element, is
    |C - C_ref| <= (4 * 2^(-8S) + 2^-21 * sqrt(steps)) * (|op(A)| |op(B)|)_ij
(plus |beta C0| * 1e-15 for the beta term, which is FP64).
"""
import numpy as np
import pytest

import oracle

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


def _bound(S, k):
    steps = S * (S + 1) // 2 * -(-k // 16)
    return 4.0 * 2.0 ** (-8 * S) + 2.0 ** -21 * np.sqrt(steps)


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (1, 1, 1), (200, 96, 130), (257, 300, 513), (64, 40, 2000)])
def test_tc_gemm_matches_oracle(B, S, ta, tb, m, n, k):
    rng = np.random.default_rng(m + 3 * n + 7 * k + S)
    A = rng.standard_normal((m, k) if ta == "N" else (k, m))
    Bm = rng.standard_normal((k, n) if tb == "N" else (n, k))
    C0 = rng.standard_normal((m, n))
    got = _host(B.purl_gemm_tc(ta, tb, _dev(A), _dev(Bm), alpha=1.5, beta=-0.5, C=_dev(C0), slices=S))
    ref = oracle.gemm(ta, tb, A, Bm, alpha=1.5, beta=-0.5, C=C0)
    mag = 1.5 * oracle.gemm(ta, tb, np.abs(A), np.abs(Bm))
    err = np.abs(got - ref)
    assert np.all(err <= _bound(S, k) * mag + 1e-15 * np.abs(C0)), (err / (mag + 1e-300)).max()


def test_tc_gemm_precision_improves_with_slices(B):
    # floating slices: 2 slices beat 1 by far; the third is capped by the
    # accumulator's rounding on this long reduction (see the module docstring)
    rng = np.random.default_rng(5)
    A, Bm = rng.standard_normal((256, 512)), rng.standard_normal((512, 192))
    ref = A @ Bm
    errs = [np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=S)) - ref).max() for S in (1, 2, 3)]
    assert errs[0] > 30 * errs[1] > 0 and errs[2] <= 1.5 * errs[1]


def test_tc_gemm_large_tile_grid(B):
    # many tiles in both directions, widest N tile, ragged edges
    rng = np.random.default_rng(6)
    m, n, k = 1000, 700, 777
    A, Bm = rng.standard_normal((m, k)), rng.standard_normal((k, n))
    got = _host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=1))
    ref = A @ Bm
    mag = np.abs(A) @ np.abs(Bm)
    assert np.all(np.abs(got - ref) <= _bound(1, k) * mag)


@pytest.mark.parametrize("S", [1, 2, 3, 4])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 64, 256), (1, 1, 1), (200, 96, 130), (257, 300, 1100), (64, 40, 3000)])
def test_tc_exact_matches_oracle(B, S, ta, tb, m, n, k):
    # fixed-point slices: the representation error of an entry is at most
    # 2^(-8S) of its row's (column's) scale 2^e_i > max_l |op(A)(i,l)|
    # (2^f_j > max_l |op(B)(l,j)|); the product error is bounded by
    # 2^(-8S+1) 2^(e_i + f_j) sqrt(k) x 4 (random signs, 4-sigma)
    rng = np.random.default_rng(m + 5 * n + 11 * k + S)
    A = rng.standard_normal((m, k) if ta == "N" else (k, m))
    Bm = rng.standard_normal((k, n) if tb == "N" else (n, k))
    opA = A if ta == "N" else A.T
    opB = Bm if tb == "N" else Bm.T
    got = _host(B.purl_gemm_tc(ta, tb, _dev(A), _dev(Bm), slices=S, exact=True))
    ref = oracle.gemm(ta, tb, A, Bm)
    ra = 2.0 ** np.ceil(np.log2(np.abs(opA).max(axis=1) + 1e-300))
    cb = 2.0 ** np.ceil(np.log2(np.abs(opB).max(axis=0) + 1e-300))
    bound = 2.0 ** (-8 * S + 1) * np.outer(ra, cb) * np.sqrt(k) * 4
    assert np.all(np.abs(got - ref) <= bound + 1e-300), (np.abs(got - ref) / bound).max()


def test_tc_exact_four_slices_reach_fp32_and_beyond(B):
    rng = np.random.default_rng(11)
    A, Bm = rng.standard_normal((300, 2048)), rng.standard_normal((2048, 200))
    ref = oracle.gemm("N", "N", A, Bm)
    err = np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=4, exact=True)) - ref).max()
    # row/column scales 2^3 each: ~2^-32 x 64 x sqrt(2048) x few
    assert err < 2.0 ** -32 * 64 * np.sqrt(2048) * 8, err


def test_tc_exact_beats_the_accumulator_floor(B):
    # the long reduction where floating slices stall at the accumulator floor
    rng = np.random.default_rng(7)
    A, Bm = rng.standard_normal((256, 4096)), rng.standard_normal((4096, 128))
    ref = oracle.gemm("N", "N", A, Bm)
    plain = np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=3)) - ref).max()
    exact = np.abs(_host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=3, exact=True)) - ref).max()
    assert exact < plain / 20, (exact, plain)
    # 3 fixed-point slices: ~2^-24 x (row scale 4) x (column scale 4) x sqrt(k) per entry
    assert exact < 2.0 ** -24 * 16 * np.sqrt(4096) * 8


def test_tc_gemm_bad_slices(B):
    with pytest.raises(B.PurlError) as e:
        B.purl_gemm_tc("N", "N", _dev(np.ones((4, 4))), _dev(np.ones((4, 4))), slices=4)
    assert e.value.status == -14
    assert B.purl_device_status() == B.PURL_OK
