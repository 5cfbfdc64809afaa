"""The C-ABI library loads and exports every entry point include/purl.h declares.

CPU-only: no call here reaches a GPU (argument checks run before any device
work), so these tests run in the no-GPU suite.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "purl.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(purl_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def purl():
    from paper_1812_06007_gb300 import build, binding
    build.build()
    return binding


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("purl_urv_factor", "purl_urv_factor_ex", "purl_urv_truncate", "purl_urv_reconstruct",
                     "purl_gaussian", "purl_qr", "purl_gemm_f64", "purl_urv_workspace_bytes",
                     "purl_status_str", "purl_device_status"):
        assert required in names


def test_every_declared_symbol_is_exported_and_bound(purl):
    L = purl.lib()
    for name in _declared():
        assert hasattr(L, name), name
        assert name in purl.SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_version(purl):
    assert purl.status_str(0) == "ok"
    assert "transpose" in purl.status_str(purl.PURL_ERR_SHAPE)
    assert purl.lib().purl_version().decode().startswith("purl")


def test_argument_errors_are_reported_before_device_work(purl):
    L = purl.lib()
    nul = ctypes.c_void_p(0)
    # m < n: shape error (factor A^T instead)
    assert L.purl_urv_factor(3, 5, nul, 3, 1, 1, 7, nul, 3, nul, 5, nul, 5, nul) == purl.PURL_ERR_SHAPE
    # LAPACK-style -i codes
    assert L.purl_urv_factor(-1, 0, nul, 1, 1, 1, 7, nul, 1, nul, 1, nul, 1, nul) == -1
    assert L.purl_urv_factor(4, 4, nul, 4, 1, 1, 7, nul, 4, nul, 4, nul, 4, nul) == -3
    fake = ctypes.c_void_p(0x1000)
    assert L.purl_urv_factor(4, 4, fake, 3, 1, 1, 7, fake, 4, fake, 4, fake, 4, nul) == -4
    assert L.purl_urv_factor(4, 4, fake, 4, -2, 1, 7, fake, 4, fake, 4, fake, 4, nul) == -5
    assert L.purl_urv_factor(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 3, fake, 4, nul) == -11
    assert L.purl_urv_factor_ex(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, 4, 99, nul, 0, nul) == -14
    assert L.purl_urv_factor_ex(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, 4, 5, nul, 0, nul) == -14
    # the FP64-emulation mode reduces over at most 2^20 rows: refused before any device work
    big = (1 << 20) + 1
    assert L.purl_urv_factor_ex(big, 4, fake, big, 1, 1, 7, fake, big, fake, 4, fake, 4, 4, nul, 0, nul) == \
        purl.PURL_ERR_UNSUPPORTED
    assert L.purl_urv_workspace_bytes(big, 4, 4) == 0
    assert L.purl_ulv_factor_ex(4, big, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, big, 4, nul, 0, nul) == \
        purl.PURL_ERR_UNSUPPORTED
    assert L.purl_qr(big, 4, fake, big, fake, big, fake, 4, 4, nul, 0, nul) == purl.PURL_ERR_UNSUPPORTED
    assert L.purl_gemm_tc(b"N", b"N", 1, 1, big, 1.0, fake, 1, fake, big, 0.0, fake, 1, 8, 1, nul) == \
        purl.PURL_ERR_UNSUPPORTED
    # exact slices: 1..4 or the FP64-emulation configuration (8); floating slices: 1..3
    for slices, exact in ((5, 1), (6, 1), (7, 1), (9, 1), (4, 0), (8, 0), (0, 1)):
        assert L.purl_gemm_tc(b"N", b"N", 1, 1, 1, 1.0, fake, 1, fake, 1, 0.0, fake, 1, slices, exact, nul) == -14
    assert L.purl_gemm_f64(b"X", b"N", 1, 1, 1, 1.0, fake, 1, fake, 1, 0.0, fake, 1, nul) == -1
    assert L.purl_urv_truncate(4, 4, 5, fake, 4, fake, 4, fake, 4, fake, 4, nul) == -3
    assert L.purl_qr(2, 3, fake, 2, fake, 2, fake, 3, 0, nul, 0, nul) == purl.PURL_ERR_SHAPE
    assert L.purl_urv_backward(3, 5, nul, 3, 1, 1, 7, nul, 3, nul, 5, nul, 5, nul, 3, nul, 0, nul) == \
        purl.PURL_ERR_SHAPE
    assert L.purl_urv_backward(4, 4, fake, 4, 1, 1, 7, nul, 4, fake, 4, fake, 4, fake, 4, nul, 0, nul) == -8
    assert L.purl_urv_backward(4, 4, fake, 4, 1, 1, 7, fake, 4, fake, 4, fake, 4, fake, 3, nul, 0, nul) == -15
    assert L.purl_urv_backward_workspace_bytes(4, 4, -1) == 0
    assert L.purl_urv_factor_batched(-1, nul, 8, 8, 1, 1, -1, nul, 0, nul) == -1
    assert L.purl_urv_factor_batched(2, nul, 8, 8, 1, 1, -1, nul, 0, nul) == -2
    assert L.purl_urv_factor_batched(0, nul, 8, 16, 1, 1, -1, nul, 0, nul) == -4
    assert L.purl_gaussian_f32(1, 0, -1, 2, nul, 1, nul) == -3
    assert L.purl_ulv_factor_ex(5, 3, fake, 5, 1, 1, 7, fake, 5, fake, 5, fake, 3, 0, nul, 0, nul) == \
        purl.PURL_ERR_SHAPE
    assert L.purl_ulv_factor_ex(3, 5, fake, 2, 1, 1, 7, fake, 3, fake, 3, fake, 5, 0, nul, 0, nul) == -4
    assert L.purl_rsvd(10, 8, fake, 10, 9, 1, 0, 7, fake, 10, fake, fake, 8, nul, 0, nul) == -5
    assert L.purl_rsvd(10, 8, fake, 10, 4, -1, 0, 7, fake, 10, fake, fake, 8, nul, 0, nul) == -6
    # empty problems are valid no-ops
    assert L.purl_urv_factor(0, 0, nul, 1, 1, 1, 7, nul, 1, nul, 1, nul, 1, nul) == 0
    assert L.purl_urv_factor(5, 0, nul, 5, 1, 1, 7, nul, 5, nul, 1, nul, 1, nul) == 0
