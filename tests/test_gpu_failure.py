"""Failure detection without a GPU fault: a bounded wait that cannot complete
(a grid barrier awaiting a block that does not exist) must come back as
PURL_ERR_TIMEOUT in the device status word, end quickly, and leave the
context usable for the next call."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def test_barrier_with_all_blocks_completes(B):
    assert B.purl_device_status() == B.PURL_OK
    B.purl_wait_probe(8, False, 1 << 16)
    assert B.purl_device_status() == B.PURL_OK


def test_barrier_missing_a_block_times_out_and_reports(B):
    import torch
    assert B.purl_device_status() == B.PURL_OK
    t0 = time.perf_counter()
    B.purl_wait_probe(4, True, 1 << 14)
    st = B.purl_device_status()  # synchronises the stream, then reads and clears
    dt = time.perf_counter() - t0
    assert st == B.PURL_ERR_TIMEOUT
    assert dt < 5.0
    assert B.purl_device_status() == B.PURL_OK  # cleared
    # the context still works: a product right after the timeout is correct
    rng = np.random.default_rng(0)
    X, Y = rng.standard_normal((70, 50)), rng.standard_normal((50, 30))
    from paper_1812_06007_gb300.binding import as_colmajor
    d = lambda a: as_colmajor(torch.from_numpy(np.asfortranarray(a)).cuda())
    C = B.purl_gemm_f64("N", "N", d(X), d(Y))
    torch.cuda.synchronize()
    assert np.abs(C.cpu().numpy() - X @ Y).max() <= 1e-12 * 50
    B.purl_wait_probe(4, False, 1 << 16)
    assert B.purl_device_status() == B.PURL_OK


def test_probe_argument_errors(B):
    import ctypes
    L = B.lib()
    nul = ctypes.c_void_p(0)
    assert L.purl_wait_probe(0, 0, 10, nul) == -1
    assert L.purl_wait_probe(4, 2, 10, nul) == -2
    assert L.purl_wait_probe(4, 0, 0, nul) == -3
