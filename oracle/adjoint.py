"""Reverse mode of PowerURV in FP64 on the CPU -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs
may import this module; it shares no code with the CUDA library.

The paper (Section 3, Eqs. (5)-(6)) defines the forward map
A -> (U, R, V) for a fixed Gaussian G but no derivative.  What this module
computes has a plain definition: the vector-Jacobian product
Abar = J(A)^T (Ubar, Rbar, Vbar), i.e. the gradient with respect to A of
<Ubar, U> + <Rbar, R> + <Vbar, V>.  It is written out as the chain rule,
step by step in the forward pass's order reversed:

  forward   Y_0 = G;  for i = 1..q:  P_i = A Y_{i-1};   Z_i = Q(P_i) if reorth else P_i
                                      W_i = A^T Z_i;     Y_i = Q(W_i) if reorth and i < q else W_i
            Y_q = V Z' (Eq. 5);   C = A V;   C = U R (Eq. 6)
  reverse   every product X = A Y contributes Abar += Xbar Y^T, Ybar = A^T Xbar
            (and X = A^T Z: Abar += Z Xbar^T, Zbar = A Xbar); every QR M = Q R
            with diag(R) > 0 maps (Qbar, Rbar) to
                Mbar = (Qbar + Q copyltu(R Rbar^T - Qbar^T Q)) R^{-T},
            copyltu(X) = tril(X) + tril(X, -1)^T (the lower triangle mirrored).

The forward products and QRs come from the FP64 oracle (``oracle.qr``, the
C Householder QR) and numpy; the triangular solve is scipy's.

``truncated_loss_grad_projection`` is a second, QR-free route to the
gradient of L(A) = ||A_k - B||_F^2 (A_k = U(:,1:k) R(1:k,:) V^T, Section 5):
by the paper's Lemma (appendix), range(U(:,1:k)) = range(A (A^T A)^q G(:,1:k)),
so A_k = P A with P the orthogonal projector onto that range, and L can be
differentiated through P = M (M^T M)^{-1} M^T, M = A (A^T A)^q G(:,1:k),
without any QR reverse rule.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import gaussian, qr


def _f64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64)


def copyltu(X: np.ndarray) -> np.ndarray:
    """tril(X) + tril(X, -1)^T: the lower triangle mirrored onto the upper one."""
    L = np.tril(X)
    return L + np.tril(X, -1).T


def qr_backward(Q, R, Qbar, Rbar=None) -> np.ndarray:
    """Mbar for M = Q R (thin QR, diag(R) > 0) given the cotangents of Q and R.

    Only the upper triangle of Rbar is used: R's strictly lower part is the
    constant zero."""
    Q, R, Qbar = _f64(Q), _f64(R), _f64(Qbar)
    n = R.shape[0]
    Rb = np.triu(_f64(Rbar)) if Rbar is not None else np.zeros((n, n))
    M = R @ Rb.T - Qbar.T @ Q
    X = Qbar + Q @ copyltu(M)
    # X R^{-T}: solve R Y^T = X^T for Y^T
    return solve_triangular(R, X.T, lower=False).T


def urv_forward_iterates(A, G, q: int, reorth: bool) -> dict:
    """Every intermediate of the forward pass (same steps as oracle.urv_g)."""
    A, G = _f64(A), _f64(G)
    Y = [G.copy()]
    Z, S, T = [], [], []
    for i in range(1, q + 1):
        P = A @ Y[i - 1]
        if reorth:
            Zi, Si = qr(P)
        else:
            Zi, Si = P, None
        Z.append(Zi)
        S.append(Si)
        W = A.T @ Zi
        if reorth and i < q:
            Yi, Ti = qr(W)
        else:
            Yi, Ti = W, None
        Y.append(Yi)
        T.append(Ti)
    V, Zp = qr(Y[q])              # Eq. 5
    U, R = qr(A @ V)              # Eq. 6
    return dict(Y=Y, Z=Z, S=S, T=T, V=V, Zp=Zp, U=U, R=R)


def urv_backward_g(A, G, q: int, reorth: bool, Ubar, Rbar, Vbar) -> np.ndarray:
    """Abar = J^T (Ubar, Rbar, Vbar) for A -> (U, R, V) with G fixed."""
    A = _f64(A)
    it = urv_forward_iterates(A, G, q, reorth)
    U, R, V, Zp = it["U"], it["R"], it["V"], it["Zp"]
    # Eq. 6: C = A V = U R
    Cbar = qr_backward(U, R, _f64(Ubar), _f64(Rbar))
    Abar = Cbar @ V.T
    Vb = _f64(Vbar) + A.T @ Cbar
    # Eq. 5: Y_q = V Z' (Z' is not an output)
    Yb = qr_backward(V, Zp, Vb, None)
    for i in range(q, 0, -1):
        Yi1, Yi, Zi = it["Y"][i - 1], it["Y"][i], it["Z"][i - 1]
        # Y_i = Q(W_i) when re-orthonormalised (i < q), else W_i
        Wb = qr_backward(Yi, it["T"][i - 1], Yb, None) if (reorth and i < q) else Yb
        # W_i = A^T Z_i
        Abar = Abar + Zi @ Wb.T
        Zb = A @ Wb
        # Z_i = Q(P_i) when re-orthonormalised, else P_i
        Pb = qr_backward(Zi, it["S"][i - 1], Zb, None) if reorth else Zb
        # P_i = A Y_{i-1}
        Abar = Abar + Pb @ Yi1.T
        Yb = A.T @ Pb
    return Abar


def urv_backward(A, q: int, reorth: bool, seed: int, Ubar, Rbar, Vbar) -> np.ndarray:
    """urv_backward_g with G = gaussian(seed, n, n) (the library's draw)."""
    n = _f64(A).shape[1]
    return urv_backward_g(A, gaussian(seed, n, n), q, reorth, Ubar, Rbar, Vbar)


def truncated_loss_cotangents(U, R, V, k: int, B):
    """L = ||U_k R_k V^T - B||^2 (U_k = U(:,1:k), R_k = R(1:k,:)): (L, Ubar, Rbar, Vbar)."""
    U, R, V, B = _f64(U), _f64(R), _f64(V), _f64(B)
    Uk, Rk = U[:, :k], R[:k, :]
    E = Uk @ Rk @ V.T - B
    Ubar = np.zeros_like(U)
    Rbar = np.zeros_like(R)
    Ubar[:, :k] = 2.0 * E @ V @ Rk.T
    Rbar[:k, :] = 2.0 * Uk.T @ E @ V
    Vbar = 2.0 * E.T @ Uk @ Rk
    return float(np.sum(E * E)), Ubar, Rbar, Vbar


def truncated_loss_grad_projection(A, G, q: int, k: int, B):
    """(L, dL/dA) for L = ||P A - B||_F^2, P the projector onto range(A (A^T A)^q G(:,1:k)).

    With M = A X_q, X_0 = G(:,1:k), X_j = A^T A X_{j-1}, and E = P A - B:
      dL = 2 <E A^T, dP> + 2 <P E, dA>,
      dP = (I - P) dM M^+ + (M^+)^T dM^T (I - P),   M^+ = R_M^{-1} Q_M^T,
    so Mbar = 2 (I - P) (E A^T + A E^T) Q_M R_M^{-T}, and Mbar is carried back
    through the products M = A X_q and X_j = A^T (A X_{j-1})."""
    A, G, B = _f64(A), _f64(G), _f64(B)
    X = [G[:, :k].copy()]
    Yp = []
    for _ in range(q):
        Yj = A @ X[-1]
        Yp.append(Yj)
        X.append(A.T @ Yj)
    M = A @ X[q]
    QM, RM = np.linalg.qr(M)
    P_of = lambda Z: QM @ (QM.T @ Z)
    E = P_of(A) - B
    L = float(np.sum(E * E))
    Abar = 2.0 * P_of(E)
    H = E @ (A.T @ QM) + A @ (E.T @ QM)
    H = H - P_of(H)
    Mbar = 2.0 * solve_triangular(RM, H.T, lower=False).T
    # M = A X_q
    Abar += Mbar @ X[q].T
    Xb = A.T @ Mbar
    for j in range(q, 0, -1):
        # X_j = A^T Y_j with Y_j = A X_{j-1}
        Abar += Yp[j - 1] @ Xb.T
        Yb = A @ Xb
        Abar += Yb @ X[j - 1].T
        Xb = A.T @ Yb
    return L, Abar
