"""Non-finite input: a NaN or an infinity in A must come back as
PURL_ERR_NONFINITE in the device status word with every output NaN, in every
mode (the tensor-core modes slice A by integer operations on its bits, which
would otherwise turn such an entry into a finite row scale and finite but
meaningless factors).  Large finite entries must not trigger the check.
Host-side only: nothing faults, the status word is read after the call."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MODES = ["fp64", "mixed", "mixed16", "emu"]


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _mode(B, name):
    return {"fp64": B.PURL_MODE_FP64, "mixed": B.PURL_MODE_MIXED_BF16, "mixed16": B.PURL_MODE_MIXED_FP16,
            "emu": B.PURL_MODE_FP64_EMU}[name]


def _dev(B, x):
    import torch
    return B.as_colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _matrix(m, n, seed=3):
    return np.random.default_rng(seed).standard_normal((m, n))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_factor_reports_nonfinite_and_returns_nan(B, mode, bad):
    assert B.purl_device_status() == B.PURL_OK
    A = _matrix(96, 80)
    A[37, 51] = bad
    U, R, V = B.purl_urv_factor(_dev(B, A), 2, True, 7, mode=_mode(B, mode))
    assert B.purl_device_status() == B.PURL_ERR_NONFINITE
    for X in (U, R, V):
        assert np.all(np.isnan(_np(X)))
    assert B.purl_device_status() == B.PURL_OK  # read and cleared
    # the next call on finite input is clean
    U, R, V = B.purl_urv_factor(_dev(B, _matrix(96, 80)), 2, True, 7, mode=_mode(B, mode))
    assert B.purl_device_status() == B.PURL_OK
    assert np.all(np.isfinite(_np(U))) and np.all(np.isfinite(_np(R))) and np.all(np.isfinite(_np(V)))


@pytest.mark.parametrize("mode", MODES)
def test_large_finite_entries_pass(B, mode):
    # large finite entries: no status, finite factors.  The mixed modes slice
    # their power-step operands with a power-of-two scale, so BF16's and
    # FP16's narrow ranges do not limit A; the Householder norms are plain
    # sums of squares, so entries are kept where their squares fit in FP64.
    scale = 1e100
    A = _matrix(72, 64) * scale
    U, R, V = B.purl_urv_factor(_dev(B, A), 1, True, 7, mode=_mode(B, mode))
    assert B.purl_device_status() == B.PURL_OK
    Un, Rn, Vn = _np(U), _np(R), _np(V)
    assert np.all(np.isfinite(Un)) and np.all(np.isfinite(Rn)) and np.all(np.isfinite(Vn))
    assert np.linalg.norm(A / scale - Un @ (Rn / scale) @ Vn.T) <= 1e-5 * np.linalg.norm(A / scale)


@pytest.mark.parametrize("mode", MODES)
def test_qr_and_ulv_report_nonfinite(B, mode):
    M = _matrix(130, 40)
    M[129, 0] = np.nan  # last row, first column: the scan's ragged tail
    Q, R = B.purl_qr(_dev(B, M), mode=_mode(B, mode))
    assert B.purl_device_status() == B.PURL_ERR_NONFINITE
    assert np.all(np.isnan(_np(Q))) and np.all(np.isnan(_np(R)))
    W = _matrix(40, 90)
    W[0, 89] = np.inf
    U, L, V = B.purl_ulv_factor_ex(_dev(B, W), 1, True, 7, mode=_mode(B, mode))
    assert B.purl_device_status() == B.PURL_ERR_NONFINITE
    for X in (U, L, V):
        assert np.all(np.isnan(_np(X)))
    assert B.purl_device_status() == B.PURL_OK


def test_rsvd_and_backward_report_nonfinite(B):
    A = _matrix(120, 100)
    A[0, 0] = np.nan
    U, S, V = B.purl_rsvd(_dev(B, A), 10, 1, 7)
    assert B.purl_device_status() == B.PURL_ERR_NONFINITE
    for X in (U, S, V):
        assert np.all(np.isnan(_np(X)))
    m, n = 64, 48
    A = _matrix(m, n)
    A[10, 47] = -np.inf
    rng = np.random.default_rng(1)
    Ub, Rb, Vb = (_dev(B, rng.standard_normal(s)) for s in ((m, n), (n, n), (n, n)))
    Ab = B.purl_urv_backward(_dev(B, A), 1, True, 7, Ub, Rb, Vb)
    assert B.purl_device_status() == B.PURL_ERR_NONFINITE
    assert np.all(np.isnan(_np(Ab)))
    assert B.purl_device_status() == B.PURL_OK
