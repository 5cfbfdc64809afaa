"""Thin ctypes binding of libpurl (``include/purl.h``); argument marshalling only.

Every function here has the C entry point's name and forwards to it; all
arithmetic runs in the library's CUDA kernels.  Tensors are torch CUDA
float64 tensors in column-major layout (``stride(0) == 1``), which is how
``empty_colmajor`` allocates them; PyTorch provides device memory and the
current stream, nothing else.  There is no CPU fallback: if ``libpurl.so`` is
missing or cannot load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpurl.so")

PURL_OK = 0
PURL_ERR_SHAPE = -100
PURL_ERR_NONFINITE = 1
PURL_ERR_TIMEOUT = 2
PURL_ERR_CUDA = 3
PURL_ERR_NOMEM = 4
PURL_ERR_UNSUPPORTED = 5
PURL_MODE_FP64 = 0
PURL_MODE_FP32 = 1
PURL_MODE_MIXED_BF16 = 2
PURL_MODE_MIXED_FP16 = 3
PURL_MODE_FP64_EMU = 4

# (name, restype, argtypes) for every symbol include/purl.h declares
_i, _u64, _d, _p, _sz, _c = (ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p,
                             ctypes.c_size_t, ctypes.c_char)
SIGNATURES = {
    "purl_status_str": (ctypes.c_char_p, [_i]),
    "purl_version": (ctypes.c_char_p, []),
    "purl_urv_factor": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _p]),
    "purl_urv_factor_ex": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_urv_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_ulv_factor_ex": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_ulv_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_rsvd": (_i, [_i, _i, _p, _i, _i, _i, _i, _u64, _p, _i, _p, _p, _i, _p, _sz, _p]),
    "purl_rsvd_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_urv_backward": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _p, _i, _p, _sz, _p]),
    "purl_urv_backward_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_urv_backward_ex": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_urv_backward_ex_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "purl_urv_factor_f32": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_urv_f32_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_urv_backward_f32": (_i, [_i, _i, _p, _i, _i, _i, _u64, _p, _i, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_urv_backward_f32_workspace_bytes": (_sz, [_i, _i, _i, _i]),
    "purl_urv_batched_variants": (_i, []),
    "purl_urv_batched_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_urv_factor_batched": (_i, [_i, _p, _i, _i, _i, _i, _i, _p, _sz, _p]),
    "purl_urv_batched_status": (_i, [_p, _p]),
    "purl_urv_batched_autotune": (_i, [_i, _p, _i, _i, _i, _i, _p, _sz, _p, ctypes.POINTER(_i),
                                       ctypes.POINTER(ctypes.c_float)]),
    "purl_gaussian_f32": (_i, [_u64, _u64, _i, _i, _p, _i, _p]),
    "purl_gaussian": (_i, [_u64, _u64, _i, _i, _p, _i, _p]),
    "purl_qr": (_i, [_i, _i, _p, _i, _p, _i, _p, _i, _i, _p, _sz, _p]),
    "purl_qr_workspace_bytes": (_sz, [_i, _i, _i]),
    "purl_gemm_f64": (_i, [_c, _c, _i, _i, _i, _d, _p, _i, _p, _i, _d, _p, _i, _p]),
    "purl_gemm_tc": (_i, [_c, _c, _i, _i, _i, _d, _p, _i, _p, _i, _d, _p, _i, _i, _i, _p]),
    "purl_gemm_tc_noalloc": (_i, [_c, _c, _i, _i, _i, _d, _p, _i, _p, _i, _d, _p, _i, _i, _p]),
    "purl_urv_truncate": (_i, [_i, _i, _i, _p, _i, _p, _i, _p, _i, _p, _i, _p]),
    "purl_urv_reconstruct": (_i, [_i, _i, _p, _i, _p, _i, _p, _i, _p, _i, _p]),
    "purl_device_status": (_i, [_p]),
    "purl_wait_probe": (_i, [_i, _i, ctypes.c_longlong, _p]),
    "purl_wait_probe_noalloc": (_i, [_i, _i, ctypes.c_longlong, _p]),
    "purl_launch_count": (ctypes.c_ulonglong, []),
    "purl_profile_enable": (None, [_i]),
    "purl_profile_reset": (None, []),
    "purl_profile_set_stride": (None, [_i]),
    "purl_profile_read": (_i, [_i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_d),
                               ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "purl_profile_class_name": (ctypes.c_char_p, [_i]),
    "purl_profile_read_named": (_i, [_i, ctypes.c_char_p, _i, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_d)]),
}

_lock = threading.Lock()
_lib = None


class PurlError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} returned {status}: {status_str(status)}")


def lib() -> ctypes.CDLL:
    """Load libpurl.so (built by ``paper_1812_06007_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1812_06007_gb300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().purl_status_str(status).decode()


def _check(fn: str, status: int):
    if status != PURL_OK:
        raise PurlError(fn, status)


# ----------------------------------------------------------- tensors ------
def _torch():
    import torch
    return torch


def empty_colmajor(rows: int, cols: int, device=None, dtype=None):
    """Uninitialised rows x cols tensor with column-major strides (1, rows)."""
    torch = _torch()
    dtype = dtype or torch.float64
    return torch.empty((cols, rows), dtype=dtype, device=device or "cuda").t()


def as_colmajor(x):
    """Column-major float64 copy of x on its device (no copy if already so)."""
    torch = _torch()
    if x.dtype != torch.float64:
        x = x.to(torch.float64)
    if x.dim() != 2:
        raise ValueError("expected a matrix")
    if x.numel() == 0 or (x.stride(0) == 1 and x.stride(1) >= max(1, x.shape[0])):
        return x
    return x.t().contiguous().t()


def _ld(x) -> int:
    if x.numel() == 0:
        return max(1, x.shape[0])
    if x.stride(0) != 1 and x.shape[0] > 1:
        raise ValueError("matrix must be column-major (stride(0) == 1)")
    return max(int(x.stride(1)), max(1, x.shape[0]))


def _cuda_check(*ts):
    torch = _torch()
    for t in ts:
        if t is not None and (not t.is_cuda or t.dtype != torch.float64):
            raise ValueError("expected CUDA float64 tensors")


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


# ------------------------------------------------------- entry points -----
def purl_gaussian(seed: int, rows: int, cols: int, stream_id: int = 0, out=None, stream=None):
    G = out if out is not None else empty_colmajor(rows, cols)
    _cuda_check(G)
    _check("purl_gaussian", lib().purl_gaussian(seed, stream_id, rows, cols, _ptr(G), _ld(G), _stream(stream)))
    return G


def purl_urv_factor(A, q: int, reorth: bool, seed: int, mode: int = PURL_MODE_FP64, out=None,
                    workspace=None, stream=None):
    """(U, R, V) with A = U R V^T by PowerURV; A is an m x n column-major CUDA float64 tensor."""
    _cuda_check(A)
    m, n = A.shape
    if out is None:
        U, R, V = empty_colmajor(m, n, A.device), empty_colmajor(n, n, A.device), empty_colmajor(n, n, A.device)
    else:
        U, R, V = out
    _cuda_check(U, R, V)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_urv_factor_ex(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(U), _ld(U), _ptr(R),
                                  _ld(R), _ptr(V), _ld(V), mode, ws_ptr, ws_bytes, _stream(stream))
    _check("purl_urv_factor_ex", st)
    return U, R, V


def purl_ulv_factor_ex(A, q: int, reorth: bool, seed: int, mode: int = PURL_MODE_FP64, workspace=None,
                       stream=None):
    """(U, L, V) with A = U L V^T for a wide A (m <= n), L lower triangular m x m."""
    _cuda_check(A)
    m, n = A.shape
    U, L, V = empty_colmajor(m, m, A.device), empty_colmajor(m, m, A.device), empty_colmajor(n, m, A.device)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_ulv_factor_ex(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(U), _ld(U), _ptr(L),
                                  _ld(L), _ptr(V), _ld(V), mode, ws_ptr, ws_bytes, _stream(stream))
    _check("purl_ulv_factor_ex", st)
    return U, L, V


def purl_rsvd(A, l: int, q: int, seed: int, reorth: bool = False, workspace=None, stream=None):
    """(U, S, V): randomized SVD A ~ U diag(S) V^T of rank l (FP64)."""
    torch = _torch()
    _cuda_check(A)
    m, n = A.shape
    U, V = empty_colmajor(m, l, A.device), empty_colmajor(n, l, A.device)
    S = torch.empty(l, dtype=torch.float64, device=A.device)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_rsvd(m, n, _ptr(A), _ld(A), l, q, int(bool(reorth)), seed, _ptr(U), _ld(U), _ptr(S), _ptr(V),
                         _ld(V), ws_ptr, ws_bytes, _stream(stream))
    _check("purl_rsvd", st)
    return U, S, V


def purl_rsvd_workspace_bytes(m: int, n: int, l: int) -> int:
    return int(lib().purl_rsvd_workspace_bytes(m, n, l))


def purl_ulv_workspace_bytes(m: int, n: int, mode: int = PURL_MODE_FP64) -> int:
    return int(lib().purl_ulv_workspace_bytes(m, n, mode))


def purl_urv_workspace_bytes(m: int, n: int, mode: int = PURL_MODE_FP64) -> int:
    return int(lib().purl_urv_workspace_bytes(m, n, mode))


def purl_urv_backward(A, q: int, reorth: bool, seed: int, Ubar, Rbar, Vbar, out=None, workspace=None,
                      stream=None):
    """Abar = J^T (Ubar, Rbar, Vbar) for the FP64 map A -> (U, R, V) of purl_urv_factor (G fixed by seed)."""
    _cuda_check(A, Ubar, Rbar, Vbar)
    m, n = A.shape
    Abar = out if out is not None else empty_colmajor(m, n, A.device)
    _cuda_check(Abar)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_urv_backward(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(Ubar), _ld(Ubar),
                                 _ptr(Rbar), _ld(Rbar), _ptr(Vbar), _ld(Vbar), _ptr(Abar), _ld(Abar), ws_ptr,
                                 ws_bytes, _stream(stream))
    _check("purl_urv_backward", st)
    return Abar


def purl_urv_backward_workspace_bytes(m: int, n: int, q: int) -> int:
    return int(lib().purl_urv_backward_workspace_bytes(m, n, q))


def purl_urv_backward_ex(A, q: int, reorth: bool, seed: int, Ubar, Rbar, Vbar, mode: int = PURL_MODE_FP64,
                         out=None, workspace=None, stream=None):
    """Abar for the map A -> (U, R, V) of purl_urv_factor_ex in `mode` (FP64, FP64_EMU or FP32)."""
    _cuda_check(A, Ubar, Rbar, Vbar)
    m, n = A.shape
    Abar = out if out is not None else empty_colmajor(m, n, A.device)
    _cuda_check(Abar)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_urv_backward_ex(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(Ubar), _ld(Ubar),
                                    _ptr(Rbar), _ld(Rbar), _ptr(Vbar), _ld(Vbar), _ptr(Abar), _ld(Abar), mode,
                                    ws_ptr, ws_bytes, _stream(stream))
    _check("purl_urv_backward_ex", st)
    return Abar


def purl_urv_backward_ex_workspace_bytes(m: int, n: int, q: int, mode: int = PURL_MODE_FP64) -> int:
    return int(lib().purl_urv_backward_ex_workspace_bytes(m, n, q, mode))


def purl_urv_f32_workspace_bytes(m: int, n: int, mode: int = PURL_MODE_FP32) -> int:
    return int(lib().purl_urv_f32_workspace_bytes(m, n, mode))


def purl_urv_backward_f32_workspace_bytes(m: int, n: int, q: int, mode: int = PURL_MODE_FP32) -> int:
    return int(lib().purl_urv_backward_f32_workspace_bytes(m, n, q, mode))


def _f32_check(*ts):
    torch = _torch()
    for t in ts:
        if t is not None and (not t.is_cuda or t.dtype != torch.float32):
            raise ValueError("expected CUDA float32 tensors")


def purl_urv_factor_f32(A, q: int, reorth: bool, seed: int, mode: int = PURL_MODE_FP32, out=None, workspace=None,
                        stream=None):
    """(U, R, V) in FP32 for a column-major CUDA float32 A (computed in `mode`, rounded once)."""
    torch = _torch()
    _f32_check(A)
    m, n = A.shape
    if out is None:
        U, R, V = (empty_colmajor(r, c, A.device, torch.float32) for r, c in ((m, n), (n, n), (n, n)))
    else:
        U, R, V = out
    _f32_check(U, R, V)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_urv_factor_f32(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(U), _ld(U), _ptr(R),
                                   _ld(R), _ptr(V), _ld(V), mode, ws_ptr, ws_bytes, _stream(stream))
    _check("purl_urv_factor_f32", st)
    return U, R, V


def purl_urv_backward_f32(A, q: int, reorth: bool, seed: int, Ubar, Rbar, Vbar, mode: int = PURL_MODE_FP32,
                          out=None, workspace=None, stream=None):
    """FP32 Abar for FP32 A and cotangents (computed in `mode`, rounded once)."""
    torch = _torch()
    _f32_check(A, Ubar, Rbar, Vbar)
    m, n = A.shape
    Abar = out if out is not None else empty_colmajor(m, n, A.device, torch.float32)
    _f32_check(Abar)
    ws_ptr, ws_bytes = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None \
        else (ctypes.c_void_p(0), 0)
    st = lib().purl_urv_backward_f32(m, n, _ptr(A), _ld(A), q, int(bool(reorth)), seed, _ptr(Ubar), _ld(Ubar),
                                     _ptr(Rbar), _ld(Rbar), _ptr(Vbar), _ld(Vbar), _ptr(Abar), _ld(Abar), mode,
                                     ws_ptr, ws_bytes, _stream(stream))
    _check("purl_urv_backward_f32", st)
    return Abar


class BatchItem(ctypes.Structure):
    """purl_batch_item of include/purl.h (64 bytes)."""
    _fields_ = [("m", _i), ("n", _i), ("lda", _i), ("ldu", _i), ("ldr", _i), ("ldv", _i),
                ("A", _p), ("U", _p), ("R", _p), ("V", _p), ("seed", _u64)]


def purl_gaussian_f32(seed: int, rows: int, cols: int, stream_id: int = 0, out=None, stream=None):
    torch = _torch()
    G = out if out is not None else empty_colmajor(rows, cols, dtype=torch.float32)
    if not G.is_cuda or G.dtype != torch.float32:
        raise ValueError("expected a CUDA float32 tensor")
    _check("purl_gaussian_f32", lib().purl_gaussian_f32(seed, stream_id, rows, cols, _ptr(G), _ld(G),
                                                        _stream(stream)))
    return G


def purl_urv_batched_variants() -> int:
    return int(lib().purl_urv_batched_variants())


def purl_urv_batched_workspace_bytes(max_m: int, max_n: int, variant: int = -1) -> int:
    return int(lib().purl_urv_batched_workspace_bytes(max_m, max_n, variant))


def purl_urv_factor_batched(items, count: int, max_m: int, max_n: int, q: int, reorth: bool, workspace,
                            variant: int = -1, stream=None):
    """items: device tensor holding `count` BatchItem records; workspace: device tensor."""
    st = lib().purl_urv_factor_batched(count, _ptr(items), max_m, max_n, q, int(bool(reorth)), variant,
                                       _ptr(workspace), workspace.numel() * workspace.element_size(),
                                       _stream(stream))
    _check("purl_urv_factor_batched", st)


def purl_urv_batched_status(workspace, stream=None) -> int:
    return int(lib().purl_urv_batched_status(_ptr(workspace), _stream(stream)))


def purl_urv_batched_autotune(items, count: int, max_m: int, max_n: int, q: int, reorth: bool, workspace,
                              stream=None):
    """(variant, ms) of the fastest variant on this batch; remembered for variant=-1 calls."""
    v = ctypes.c_int(-1)
    ms = ctypes.c_float(0.0)
    st = lib().purl_urv_batched_autotune(count, _ptr(items), max_m, max_n, q, int(bool(reorth)), _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), _stream(stream),
                                         ctypes.byref(v), ctypes.byref(ms))
    _check("purl_urv_batched_autotune", st)
    return v.value, ms.value


def purl_qr(M, mode: int = PURL_MODE_FP64, want_q: bool = True, want_r: bool = True, stream=None):
    """Q, R with M = Q R, diag(R) >= 0 (unpivoted Householder QR on the GPU)."""
    _cuda_check(M)
    m, n = M.shape
    Q = empty_colmajor(m, n, M.device) if want_q else None
    R = empty_colmajor(n, n, M.device) if want_r else None
    st = lib().purl_qr(m, n, _ptr(M), _ld(M), _ptr(Q), _ld(Q) if Q is not None else 1, _ptr(R),
                       _ld(R) if R is not None else 1, mode, ctypes.c_void_p(0), 0, _stream(stream))
    _check("purl_qr", st)
    return Q, R


def purl_gemm_f64(transa: str, transb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None,
                  stream=None):
    _cuda_check(A, B)
    m = A.shape[0] if transa == "N" else A.shape[1]
    k = A.shape[1] if transa == "N" else A.shape[0]
    n = B.shape[1] if transb == "N" else B.shape[0]
    if C is None:
        C = empty_colmajor(m, n, A.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
    _cuda_check(C)
    st = lib().purl_gemm_f64(transa.encode(), transb.encode(), m, n, k, alpha, _ptr(A), _ld(A), _ptr(B),
                             _ld(B), beta, _ptr(C), _ld(C), _stream(stream))
    _check("purl_gemm_f64", st)
    return C


def purl_gemm_tc(transa: str, transb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None,
                 slices: int = 3, exact: bool = False, stream=None):
    """C = alpha op(A) op(B) + beta C on the BF16 tensor cores with `slices` BF16 slices per operand."""
    _cuda_check(A, B)
    m = A.shape[0] if transa == "N" else A.shape[1]
    k = A.shape[1] if transa == "N" else A.shape[0]
    n = B.shape[1] if transb == "N" else B.shape[0]
    if C is None:
        C = empty_colmajor(m, n, A.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
    _cuda_check(C)
    st = lib().purl_gemm_tc(transa.encode(), transb.encode(), m, n, k, alpha, _ptr(A), _ld(A), _ptr(B),
                            _ld(B), beta, _ptr(C), _ld(C), slices, int(bool(exact)), _stream(stream))
    _check("purl_gemm_tc", st)
    return C


def purl_gemm_tc_noalloc(transa: str, transb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None,
                         slices: int = 3, stream=None):
    """purl_gemm_tc (floating slices) staged in the library's static device scratch: allocates nothing."""
    _cuda_check(A, B)
    m = A.shape[0] if transa == "N" else A.shape[1]
    k = A.shape[1] if transa == "N" else A.shape[0]
    n = B.shape[1] if transb == "N" else B.shape[0]
    if C is None:
        C = empty_colmajor(m, n, A.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
    _cuda_check(C)
    st = lib().purl_gemm_tc_noalloc(transa.encode(), transb.encode(), m, n, k, alpha, _ptr(A), _ld(A), _ptr(B),
                                    _ld(B), beta, _ptr(C), _ld(C), slices, _stream(stream))
    _check("purl_gemm_tc_noalloc", st)
    return C


def purl_urv_truncate(U, R, V, k: int, out=None, stream=None):
    _cuda_check(U, R, V)
    m, n = U.shape
    Ak = out if out is not None else empty_colmajor(m, n, U.device)
    st = lib().purl_urv_truncate(m, n, k, _ptr(U), _ld(U), _ptr(R), _ld(R), _ptr(V), _ld(V), _ptr(Ak),
                                 _ld(Ak), _stream(stream))
    _check("purl_urv_truncate", st)
    return Ak


def purl_urv_reconstruct(U, R, V, out=None, stream=None):
    _cuda_check(U, R, V)
    m, n = U.shape
    Ak = out if out is not None else empty_colmajor(m, n, U.device)
    st = lib().purl_urv_reconstruct(m, n, _ptr(U), _ld(U), _ptr(R), _ld(R), _ptr(V), _ld(V), _ptr(Ak),
                                    _ld(Ak), _stream(stream))
    _check("purl_urv_reconstruct", st)
    return Ak


def purl_wait_probe(blocks: int, missing: bool, polls: int, stream=None):
    _check("purl_wait_probe", lib().purl_wait_probe(blocks, int(bool(missing)), polls, _stream(stream)))


def purl_wait_probe_noalloc(blocks: int, missing: bool, polls: int, stream=None):
    _check("purl_wait_probe_noalloc",
           lib().purl_wait_probe_noalloc(blocks, int(bool(missing)), polls, _stream(stream)))


def purl_device_status(stream=None) -> int:
    return int(lib().purl_device_status(_stream(stream)))


def purl_launch_count() -> int:
    return int(lib().purl_launch_count())


def purl_profile_enable(on: bool = True):
    lib().purl_profile_enable(int(bool(on)))


def purl_profile_set_stride(stride: int):
    lib().purl_profile_set_stride(stride)


def purl_profile_reset():
    lib().purl_profile_reset()


PROFILE_CLASSES = ("gemm_f64", "panel_qr", "gemm_tc", "split", "other")


def purl_profile_read() -> dict:
    """{class name: {launches, ms, flops, bytes}} since the last reset (synchronises)."""
    out = {}
    for cls, name in enumerate(PROFILE_CLASSES):
        n = ctypes.c_longlong(0)
        ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        lib().purl_profile_read(cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by))
        out[name] = {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}
    return out


def purl_profile_read_named() -> dict:
    """{kernel name: {launches, ms}} since the last reset (synchronises)."""
    out = {}
    i = 0
    while True:
        buf = ctypes.create_string_buffer(128)
        n = ctypes.c_longlong(0)
        ms, fl, by = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        if lib().purl_profile_read_named(i, buf, 128, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                         ctypes.byref(by)) != 0:
            break
        out[buf.value.decode()] = {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}
        i += 1
    return out
