"""Seeded synthetic inputs shaped like the paper's test matrices (Section 5).

This module holds input synthesis only -- none of the PowerURV arithmetic.
Both the CUDA path's tests/benchmarks and the FP64 oracle take their inputs
from here, so that the two sides factor byte-identical matrices.

Test matrices follow the recipe of Section 5: A = Uh diag(sigma) Vh^T with
Uh, Vh Haar-distributed orthogonal factors.  A Haar factor is the Q of a QR
of a seeded N(0,1) matrix with the signs fixed so that diag(R) > 0 (the
footnote of Section 2.2 explains why the sign fix is needed for Haar).  The
QR here is numpy's LAPACK (host) or torch's (device) -- a library routine
used for input synthesis, never the code under test.

sigma profiles:
  exponential  sigma_j = 10^(-d (j-1)/(n-1))     (decay to 10^-d)
  polynomial   sigma_j = j^-p                     (Matrix 2 uses p = 1)
  step         sigma_j = 1 for j <= n/4, else h
"""
from __future__ import annotations

import numpy as np

# Seeds used throughout the tests and the benchmark.
SEED_U = 1001   # left Haar factor
SEED_V = 1002   # right Haar factor
SEED_G = 7      # PowerURV's Gaussian start matrix (Philox key)
SEED_B = 9      # target matrix of the adjoint loss


def sigma_profile(kind: str, n: int, decades: float = 8.0, power: float = 2.0,
                  low: float = 1e-6) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    if kind == "exponential":
        return 10.0 ** (-decades * (j - 1) / max(n - 1, 1))
    if kind == "polynomial":
        return j ** (-power)
    if kind == "step":
        return np.where(j <= n / 4, 1.0, low)
    raise ValueError(f"unknown sigma profile {kind!r}")


def haar_np(rows: int, cols: int, seed: int) -> np.ndarray:
    """rows x cols matrix with Haar-distributed orthonormal columns (rows >= cols)."""
    X = np.random.default_rng(seed).standard_normal((rows, cols))
    Q, R = np.linalg.qr(X)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d)


def test_matrix_np(m: int, n: int, sigma: np.ndarray, seed_u: int = SEED_U,
                   seed_v: int = SEED_V) -> np.ndarray:
    """A = Uh diag(sigma) Vh^T, m x n, column-major float64 (host)."""
    Uh = haar_np(m, n, seed_u)
    Vh = haar_np(n, n, seed_v)
    return np.asfortranarray((Uh * sigma) @ Vh.T)


def gaussian_matrix_np(m: int, n: int, seed: int) -> np.ndarray:
    """Gaussian-entry A (Section 4's timing matrices), column-major float64."""
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((m, n)))


def _haar_torch(rows: int, cols: int, seed: int, device, dtype):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    X = torch.randn(rows, cols, generator=gen, device=device, dtype=dtype)
    Q, R = torch.linalg.qr(X)
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return Q * d


def test_matrix_torch(m: int, n: int, sigma, seed_u: int = SEED_U, seed_v: int = SEED_V,
                      device="cuda", qr_dtype=None):
    """A = Uh diag(sigma) Vh^T built on `device` (for sizes too large for the host).

    Returns a float64 tensor holding A in column-major order: the tensor is the
    transpose-view of a row-major n x m buffer, so ``A.t().contiguous()`` is not
    needed by callers that pass ``A.data_ptr()`` with lda = m.  The Haar factors
    are drawn with torch's generator, so these matrices differ from
    ``test_matrix_np`` for the same seeds; the sigma profile is the same.
    ``qr_dtype`` (default float64) may be float32 to speed up synthesis of very
    large inputs; A is then orthogonally mixed only to ~1e-6, which changes its
    singular values by that relative amount and nothing else.
    """
    import torch
    qr_dtype = qr_dtype or torch.float64
    s = torch.as_tensor(np.asarray(sigma), device=device, dtype=torch.float64)
    Uh = _haar_torch(m, n, seed_u, device, qr_dtype).to(torch.float64)
    Vh = _haar_torch(n, n, seed_v, device, qr_dtype).to(torch.float64)
    A_rowmajor = (Uh * s) @ Vh.t()             # m x n, row-major
    del Uh, Vh
    # column-major m x n storage == row-major n x m storage of A^T
    return A_rowmajor.t().contiguous().t()


def gaussian_matrix_torch(m: int, n: int, seed: int, device="cuda"):
    """Gaussian-entry m x n float64 tensor in column-major storage."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randn(n, m, generator=gen, device=device, dtype=torch.float64).t()
