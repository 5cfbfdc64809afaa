"""Seeded synthetic inputs shaped like the paper's test matrices (Section 5).

This module holds input synthesis only -- none of the PowerURV arithmetic.
Both the CUDA path's tests/benchmarks and the FP64 oracle take their inputs
from here, so that the two sides factor byte-identical matrices.

Test matrices follow the recipe of Section 5: A = Uh diag(sigma) Vh^T with
Uh, Vh Haar-distributed orthogonal factors.  A Haar factor is the Q of a QR
of a seeded N(0,1) matrix with the signs fixed so that diag(R) > 0 (the
footnote of Section 2.2 explains why the sign fix is needed for Haar).  The
QR here is numpy's LAPACK on the host -- a library routine used for input
synthesis, never the code under test.  Inputs too large for a host QR use
MixedOrthogonal factors (see below).

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
SEED_BATCH = 10000  # batched matrix i: Haar factors and G keyed by SEED_BATCH + i


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


# Matrices 1-3 of the paper's numerical section (200 x 160, Haar factors).
QUALITY_M, QUALITY_N = 200, 160
QUALITY_SEED_U, QUALITY_SEED_V = 71, 72


def quality_sigma(name: str, n: int = QUALITY_N) -> np.ndarray:
    """Singular values of the paper's test matrices (Section 7), with these readings:
    "fast": Matrix 1, printed as (1e-20)^(k-1), which underflows after k ~ 16; read as
            10^(-20 (k-1)/(n-1)), twenty decades over the n values;
    "slow": Matrix 2, 1/k;
    "s":    Matrix 3, 10^-(1 + tanh(5(-1 + 2k/n))) for k <= 80 with n = 160, and 10^-2 for every
            k > 80 (the text gives 81..150 only)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    if name == "fast":
        return 10.0 ** (-20.0 * (k - 1) / max(n - 1, 1))
    if name == "slow":
        return 1.0 / k
    if name == "s":
        return np.where(k <= 80, 10.0 ** (-(1.0 + np.tanh(5.0 * (-1.0 + 2.0 * k / n)))), 1e-2)
    raise ValueError(f"unknown test matrix {name!r}")


def quality_matrix_np(name: str) -> np.ndarray:
    """Matrix 1, 2 or 3 ("fast", "slow", "s"): Uh diag(sigma) Vh^T, 200 x 160."""
    return test_matrix_np(QUALITY_M, QUALITY_N, quality_sigma(name, QUALITY_N), QUALITY_SEED_U, QUALITY_SEED_V)


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


class MixedOrthogonal:
    """Dense orthogonal N x N operator M = B1 P B2 for inputs too large for a
    host QR: B1, B2 block-diagonal with Haar blocks (host numpy QR of seeded
    Gaussian blocks, sign-fixed), P a seeded row permutation.  Every row of M
    mixes every block, M is orthogonal to rounding, and it is applied in
    O(N^2 nb) work instead of being formed.  It is not exactly Haar
    distributed; the benchmark uses it only where the spectrum, not the
    distribution of the singular vectors, matters."""

    def __init__(self, N: int, seed: int, nb: int = 1024):
        rng = np.random.default_rng(seed)
        self.N, self.nb = N, nb
        self.sizes = [min(nb, N - s) for s in range(0, N, nb)]
        self.B1 = [haar_np(b, b, int(rng.integers(1 << 62))) for b in self.sizes]
        self.B2 = [haar_np(b, b, int(rng.integers(1 << 62))) for b in self.sizes]
        self.perm = rng.permutation(N)

    def apply(self, X):
        """M @ X for a torch float64 tensor X (N x k) on any device."""
        import torch
        dev = X.device

        def blockdiag(Bs, Y):
            out = torch.empty_like(Y)
            r = 0
            for B in Bs:
                b = B.shape[0]
                out[r:r + b] = torch.as_tensor(B, device=dev) @ Y[r:r + b]
                r += b
            return out

        Y = blockdiag(self.B2, X)
        Y = Y[torch.as_tensor(self.perm, device=dev)]
        return blockdiag(self.B1, Y)


def test_matrix_torch(m: int, n: int, sigma, seed_u: int = SEED_U, seed_v: int = SEED_V,
                      device="cuda", nb: int = 1024):
    """A = Uh diag(sigma) Vh^T (m x n, float64, column-major) built on `device`.

    Uh is the first n columns of a MixedOrthogonal(m), Vh a MixedOrthogonal(n),
    so A has exactly the singular values sigma (to rounding).  Uses only
    matrix products on the device (no device linear-algebra library).
    """
    import torch
    s = torch.as_tensor(np.asarray(sigma), device=device, dtype=torch.float64)
    Mv = MixedOrthogonal(n, seed_v, nb)
    Vt = Mv.apply(torch.eye(n, dtype=torch.float64, device=device)).t().contiguous()  # Vh^T
    C = torch.zeros((m, n), dtype=torch.float64, device=device)
    C[:n] = s[:, None] * Vt                       # [diag(sigma) Vh^T ; 0]
    del Vt
    A_rowmajor = MixedOrthogonal(m, seed_u, nb).apply(C)   # Mu [diag(sigma) Vh^T; 0]
    del C
    return A_rowmajor.t().contiguous().t()


def gaussian_matrix_torch(m: int, n: int, seed: int, device="cuda"):
    """Gaussian-entry m x n float64 tensor in column-major storage."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randn(n, m, generator=gen, device=device, dtype=torch.float64).t()


# ------------------------------------------------------------ batched ------
def batched_shapes(count: int, seed: int = SEED_BATCH, n_lo: int = 16, n_hi: int = 256):
    """Sizes of the batched workload: n ~ U[n_lo, n_hi], m ~ U[n, 2n] (integers)."""
    rng = np.random.default_rng(seed)
    n = rng.integers(n_lo, n_hi + 1, size=count)
    m = np.array([int(rng.integers(k, 2 * k + 1)) for k in n], dtype=np.int64)
    return m.astype(np.int64), n.astype(np.int64)


def _haar_gen(rng, rows: int, cols: int) -> np.ndarray:
    Q, R = np.linalg.qr(rng.standard_normal((rows, cols)))
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def batched_matrix_np(m: int, n: int, index: int, decades: float = 6.0) -> np.ndarray:
    """Matrix `index` of the batch: Uh diag(10^(-decades (j-1)/(n-1))) Vh^T in
    FP32 (column-major), Uh (m x n) and Vh (n x n) Haar with seeds derived
    from SEED_BATCH + index."""
    key = SEED_BATCH + index
    Uh = _haar_gen(np.random.default_rng([key, 1]), m, n)
    Vh = _haar_gen(np.random.default_rng([key, 2]), n, n)
    sig = 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))
    return np.asfortranarray(((Uh * sig) @ Vh.T).astype(np.float32))


def batched_seed(index: int) -> int:
    """Philox key of matrix `index`'s Gaussian start matrix G."""
    return SEED_BATCH + index
