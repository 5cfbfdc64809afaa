"""Randomized SVD (Section 6 of the paper) in FP64 on the CPU -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs
may import this module; it shares no code with the CUDA library.

The steps are the paper's Eqs. (rsvd1)-(rsvd4), in their order:
  G_rsvd = G(:, 1:l)                       (the first l columns of PowerURV's G)
  Y      = A (A^T A)^q G_rsvd              (rsvd1; with `reorth`, the iterate is
                                            replaced by the Q of its QR after every
                                            product, as in the PowerURV oracle)
  Y      = Q R                             (rsvd2, unpivoted Householder QR, diag(R) >= 0)
  Q^T A  = W Sigma V^T                     (rsvd3, a deterministic SVD; numpy's
                                            LAPACK SVD serves as that step)
  U      = Q W                             (rsvd4)
The SVD's signs are fixed by one convention, shared with the library: in
every column of U the entry of largest magnitude (the first one on ties) is
positive, and the matching column of V is flipped with it.
"""
from __future__ import annotations

import numpy as np

from . import gaussian, qr


def _f64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


def fix_signs(U: np.ndarray, V: np.ndarray):
    """Flip U(:, j), V(:, j) so that U's largest-magnitude entry of column j is positive."""
    U, V = U.copy(), V.copy()
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0:
            U[:, j] = -U[:, j]
            V[:, j] = -V[:, j]
    return U, V


def range_basis(A, G, q: int, reorth: bool) -> np.ndarray:
    """Q_rsvd of Eqs. (rsvd1)-(rsvd2): orthonormal basis of A (A^T A)^q G."""
    A, X = _f64(A), _f64(G)
    for _ in range(q):
        P = A @ X
        if reorth:
            P, _ = qr(P)
        X = A.T @ P
        if reorth:
            X, _ = qr(X)
    Q, _ = qr(A @ X)
    return Q


def rsvd_g(A, G, q: int, reorth: bool = False):
    """(U, sigma, V) of the RSVD started from the n x l matrix G."""
    A = _f64(A)
    Q = range_basis(A, G, q, reorth)
    W, s, Vt = np.linalg.svd(Q.T @ A, full_matrices=False)
    U, V = fix_signs(Q @ W, Vt.T)
    return U, s, V


def rsvd(A, l: int, q: int, seed: int, reorth: bool = False):
    """RSVD with G_rsvd = the first l columns of gaussian(seed, n, n)."""
    n = _f64(A).shape[1]
    return rsvd_g(A, gaussian(seed, n, l), q, reorth)
