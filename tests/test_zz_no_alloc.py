"""The allocation-free product entry point (purl_gemm_tc_noalloc), through the C ABI.

Some callers cannot allocate device memory when they call the library (their
framework's caching allocator already owns the GPU, or their loop forbids
allocation); purl_gemm_tc_noalloc stages its operand slices in a fixed
24 MiB device array instead.  It must give what the allocating entry point
purl_gemm_tc gives, call after call (the array is reused), within the same
tolerance as the tensor-core product tests.  This file is collected last so
that a stop at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes

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
    # same bound as the tensor-core product tests (test_gpu_tc.py)
    steps = S * (S + 1) // 2 * -(-k // 16)
    return 4.0 * 2.0 ** (-8 * S) + 2.0 ** -21 * np.sqrt(steps)


@pytest.mark.parametrize("S", [1, 3])
@pytest.mark.parametrize("ta,tb,m,n,k", [("N", "N", 300, 200, 150), ("T", "N", 129, 77, 513), ("N", "T", 64, 300, 96)])
def test_noalloc_matches_allocating_entry_on_consecutive_calls(B, S, ta, tb, m, n, k):
    rng = np.random.default_rng(m + n + k + S)
    for call in range(2):  # the static scratch keeps the previous call's contents
        A = rng.standard_normal((m, k) if ta == "N" else (k, m))
        Bm = rng.standard_normal((k, n) if tb == "N" else (n, k))
        C0 = rng.standard_normal((m, n))
        got = _host(B.purl_gemm_tc_noalloc(ta, tb, _dev(A), _dev(Bm), alpha=0.5, beta=2.0, C=_dev(C0), slices=S))
        ref = _host(B.purl_gemm_tc(ta, tb, _dev(A), _dev(Bm), alpha=0.5, beta=2.0, C=_dev(C0), slices=S))
        mag = 0.5 * oracle.gemm(ta, tb, np.abs(A), np.abs(Bm))
        assert np.all(np.abs(got - ref) <= _bound(S, k) * mag + 1e-14 * np.abs(C0)), (call, np.abs(got - ref).max())
        exact = oracle.gemm(ta, tb, A, Bm, alpha=0.5, beta=2.0, C=C0)
        assert np.all(np.abs(got - exact) <= _bound(S, k) * mag + 1e-14 * np.abs(C0))
    assert B.purl_device_status() == B.PURL_OK


def test_noalloc_timeout_reaches_device_status(B):
    # A bounded wait that runs out while reporting to the no-alloc array's own
    # status word (a grid barrier that awaits one block too many, short poll
    # limit) must come back through purl_device_status and then be cleared.
    assert B.purl_device_status() == B.PURL_OK
    B.purl_wait_probe_noalloc(4, True, 1 << 14)
    assert B.purl_device_status() == B.PURL_ERR_TIMEOUT
    assert B.purl_device_status() == B.PURL_OK
    # the entry point still gives the allocating entry point's result afterwards
    rng = np.random.default_rng(5)
    A, Bm = rng.standard_normal((96, 80)), rng.standard_normal((80, 40))
    got = _host(B.purl_gemm_tc_noalloc("N", "N", _dev(A), _dev(Bm), slices=2))
    ref = _host(B.purl_gemm_tc("N", "N", _dev(A), _dev(Bm), slices=2))
    assert np.all(np.abs(got - ref) <= _bound(2, 80) * np.abs(A) @ np.abs(Bm))
    assert B.purl_device_status() == B.PURL_OK


def test_noalloc_rejects_requests_beyond_its_scratch(B):
    import torch
    L = B.lib()
    # 2 * 3 slices * 4096 * (4096 + 4096) bytes = 192 MiB > 24 MiB: refused before any work
    A = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    nul = ctypes.c_void_p(A.data_ptr())
    st = L.purl_gemm_tc_noalloc(b"N", b"N", 4096, 4096, 4096, 1.0, nul, 4096, nul, 4096, 0.0, nul, 4096, 3,
                                ctypes.c_void_p(0))
    assert st == B.PURL_ERR_NOMEM
    # k = 0 scales C by beta without touching the scratch
    C = _dev(np.ones((5, 4)))
    B.purl_gemm_tc_noalloc("N", "N", _dev(np.ones((5, 0))), _dev(np.ones((0, 4))), alpha=1.0, beta=3.0, C=C, slices=1)
    assert np.all(_host(C) == 3.0)
