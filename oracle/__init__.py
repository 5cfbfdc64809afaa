"""FP64 CPU oracle for PowerURV (arXiv:1812.06007) -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the GPU
library is checked against.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA library (``paper_1812_06007_gb300``) and imports nothing from it.

The arithmetic lives in ``purl_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that x86-64 and AArch64 agree bit for bit).  This
module only compiles it on first use and marshals numpy arrays through ctypes.
All matrices are column-major (numpy ``order='F'``) float64.

Paper map (sections / equations of the paper):
  gaussian      Section 3, the Gaussian test matrix G (Philox4x64-10 + Box-Muller;
                the generator is this project's choice, the paper names none)
  qr            Section 2.2, unpivoted Householder QR, diag(R) >= 0
  urv / urv_g   Section 3, Eq. (5) and Eq. (6), re-orthonormalisation in the
                power iteration (Section 3, third paragraph); q = 0 is DDH-URV
  ulv           Section 1, the wide case: the URV of A^T read as A = U L V^T
  truncate      Section 5, A_k = U(:,1:k) R(1:k,:) V^T
  jacobi_svd    brute-force singular values for tiny inputs (tests only)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "purl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libpurl_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O3", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile purl_oracle.c into libpurl_oracle.so (next to the source)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, u64, dbl, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.orc_philox4x64_10.argtypes = [p, p, p]
            lib.orc_uniforms.argtypes = [u64, u64, i64, p]
            lib.orc_gaussian.argtypes = [u64, u64, i64, i64, p, i64]
            lib.orc_gemm.argtypes = [ctypes.c_char, ctypes.c_char, i64, i64, i64, dbl, p, i64, p, i64, dbl, p, i64]
            lib.orc_householder_qr.argtypes = [i64, i64, p, i64, p]
            lib.orc_form_q.argtypes = [i64, i64, p, i64, p, p, i64]
            lib.orc_qr_explicit.argtypes = [i64, i64, p, i64, p, i64, p, i64]
            lib.orc_qr_explicit.restype = ctypes.c_int
            lib.orc_urv_factor_g.argtypes = [i64, i64, p, i64, p, i64, ctypes.c_int, ctypes.c_int,
                                             p, i64, p, i64, p, i64]
            lib.orc_urv_factor_g.restype = ctypes.c_int
            lib.orc_urv_factor.argtypes = [i64, i64, p, i64, ctypes.c_int, ctypes.c_int, u64,
                                           p, i64, p, i64, p, i64]
            lib.orc_urv_factor.restype = ctypes.c_int
            lib.orc_truncate.argtypes = [i64, i64, i64, p, i64, p, i64, p, i64, p, i64]
            lib.orc_truncate.restype = ctypes.c_int
            lib.orc_jacobi_svd.argtypes = [i64, i64, p, i64, p]
            lib.orc_jacobi_svd.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x64_10(counter, key) -> np.ndarray:
    """One Philox4x64-10 block: 4 uint64 words for counter (4 words), key (2 words)."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniforms(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """The uniform (0,1) stream behind gaussian(): element e is word e%4 of block e/4."""
    u = np.zeros(max(count, 1), dtype=np.float64)
    _load().orc_uniforms(seed, stream, count, _ptr(u))
    return u[:count]


def gaussian(seed: int, rows: int, cols: int, stream: int = 0) -> np.ndarray:
    """N(0,1) matrix (rows x cols, column-major) for (seed, stream)."""
    G = np.zeros((rows, cols), dtype=np.float64, order="F")
    if rows * cols:
        _load().orc_gaussian(seed, stream, rows, cols, _ptr(G), max(rows, 1))
    return G


def gemm(ta: str, tb: str, A, B, alpha: float = 1.0, beta: float = 0.0, C=None) -> np.ndarray:
    """C = alpha op(A) op(B) + beta C by definition (one dot product per entry)."""
    A, B = _f64(A), _f64(B)
    m = A.shape[0] if ta == "N" else A.shape[1]
    k = A.shape[1] if ta == "N" else A.shape[0]
    n = B.shape[1] if tb == "N" else B.shape[0]
    C = np.zeros((m, n), order="F") if C is None else _f64(C).copy(order="F")
    _load().orc_gemm(ta.encode(), tb.encode(), m, n, k, alpha, _ptr(A), max(A.shape[0], 1),
                     _ptr(B), max(B.shape[0], 1), beta, _ptr(C), max(m, 1))
    return C


def householder_qr(A):
    """Raw unpivoted Householder QR: (packed factor, tau), LAPACK-style storage."""
    F = _f64(A).copy(order="F")
    m, n = F.shape
    tau = np.zeros(max(min(m, n), 1))
    _load().orc_householder_qr(m, n, _ptr(F), max(m, 1), _ptr(tau))
    return F, tau[: min(m, n)]


def qr(M):
    """Q (m x n), R (n x n) with M = Q R and diag(R) >= 0 (m >= n)."""
    M = _f64(M)
    m, n = M.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    rc = _load().orc_qr_explicit(m, n, _ptr(M), max(m, 1), _ptr(Q), max(m, 1), _ptr(R), max(n, 1))
    if rc != 0:
        raise ValueError(f"orc_qr_explicit failed ({rc}); need m >= n")
    return Q, R


def urv_g(A, G, q: int, reorth: bool):
    """PowerURV from an explicit starting matrix G: returns (U, R, V), A = U R V^T."""
    A, G = _f64(A), _f64(G)
    m, n = A.shape
    U = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    V = np.zeros((n, n), order="F")
    rc = _load().orc_urv_factor_g(m, n, _ptr(A), max(m, 1), _ptr(G), max(n, 1), q, int(bool(reorth)),
                                  _ptr(U), max(m, 1), _ptr(R), max(n, 1), _ptr(V), max(n, 1))
    if rc != 0:
        raise ValueError(f"orc_urv_factor_g failed ({rc})")
    return U, R, V


def urv(A, q: int, reorth: bool, seed: int):
    """PowerURV with G = gaussian(seed, n, n): returns (U, R, V), A = U R V^T."""
    A = _f64(A)
    m, n = A.shape
    U = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    V = np.zeros((n, n), order="F")
    rc = _load().orc_urv_factor(m, n, _ptr(A), max(m, 1), q, int(bool(reorth)), seed,
                                _ptr(U), max(m, 1), _ptr(R), max(n, 1), _ptr(V), max(n, 1))
    if rc != 0:
        raise ValueError(f"orc_urv_factor failed ({rc})")
    return U, R, V


def ulv(A, q: int, reorth: bool, seed: int):
    """Wide A (m <= n): (U, L, V) with A = U L V^T, L lower triangular (m x m).

    Section 1: a URV factorization of A^T gives a ULV factorization of A.
    With A^T = U' R' V'^T (PowerURV of the n x m matrix A^T, G m x m from
    `seed`): U = V', L = R'^T, V = U'."""
    A = _f64(A)
    m, n = A.shape
    if m > n:
        raise ValueError("ulv needs m <= n")
    Up, Rp, Vp = urv(np.asfortranarray(A.T), q, reorth, seed)
    return np.asfortranarray(Vp), np.asfortranarray(Rp.T), np.asfortranarray(Up)


def truncate(U, R, V, k: int) -> np.ndarray:
    """A_k = U(:,1:k) R(1:k,:) V^T."""
    U, R, V = _f64(U), _f64(R), _f64(V)
    m, n = U.shape
    Ak = np.zeros((m, n), order="F")
    rc = _load().orc_truncate(m, n, k, _ptr(U), max(m, 1), _ptr(R), max(n, 1), _ptr(V), max(n, 1),
                              _ptr(Ak), max(m, 1))
    if rc != 0:
        raise ValueError(f"orc_truncate failed ({rc})")
    return Ak


def jacobi_svd(A) -> np.ndarray:
    """Singular values (decreasing) by one-sided Jacobi; for tiny inputs only."""
    A = _f64(A)
    m, n = A.shape
    s = np.zeros(max(n, 1))
    _load().orc_jacobi_svd(m, n, _ptr(A), max(m, 1), _ptr(s))
    return s[:n]
