"""Pins of the oracle's reverse mode (oracle.adjoint) against facts that do not
come from the oracle's own chain rule:

* central finite differences of the forward oracle (the C PowerURV of
  Section 3, itself pinned in test_oracle.py),
* the composite identity: with k = n, A_k = U R V^T = A for every G, so
  L = ||A_k - B||^2 has gradient exactly 2 (A - B),
* the appendix Lemma: range(U(:,1:k)) = range(A (A^T A)^q G(:,1:k)), which
  gives a QR-free formula for the gradient of the truncated loss,
* q = 0: V = Q(G) does not depend on A, so Vbar cannot change Abar.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint


def _haar(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def _wellcond(seed, m, n, lo=0.3):
    """U diag(sigma) V^T with sigma spaced in [lo, 1]: condition number 1/lo."""
    rng = np.random.default_rng(seed)
    Uh = _haar(rng, m)[:, :n]
    Vh = _haar(rng, n)
    s = np.linspace(1.0, lo, n)
    return np.asfortranarray((Uh * s) @ Vh.T)


def _fd_directional(f, A, D, h):
    return (f(A + h * D) - f(A - h * D)) / (2.0 * h)


# ---------------------------------------------------------------- QR rule --
@pytest.mark.parametrize("m,n", [(8, 5), (6, 6), (13, 4)])
def test_qr_backward_matches_finite_differences(m, n):
    rng = np.random.default_rng(100 + m * 10 + n)
    M = rng.standard_normal((m, n)) + 2.0 * np.eye(m, n)
    Qbar = rng.standard_normal((m, n))
    Rbar = np.triu(rng.standard_normal((n, n)))

    def f(X):
        Q, R = oracle.qr(X)
        return float(np.sum(Qbar * Q) + np.sum(Rbar * R))

    Mbar = adjoint.qr_backward(*oracle.qr(M), Qbar, Rbar)
    for t in range(4):
        D = rng.standard_normal((m, n))
        fd = _fd_directional(f, M, D, 1e-6)
        an = float(np.sum(Mbar * D))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (t, fd, an)


def test_qr_backward_ignores_lower_triangle_of_rbar():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((9, 6))
    Q, R = oracle.qr(M)
    Qbar = rng.standard_normal((9, 6))
    Rbar = rng.standard_normal((6, 6))
    a = adjoint.qr_backward(Q, R, Qbar, Rbar)
    b = adjoint.qr_backward(Q, R, Qbar, np.triu(Rbar))
    assert np.array_equal(a, b)


def test_copyltu_mirrors_lower_triangle():
    X = np.arange(16.0).reshape(4, 4)
    Y = adjoint.copyltu(X)
    assert np.array_equal(np.tril(Y), np.tril(X))
    assert np.array_equal(Y, Y.T)


# ------------------------------------------------------ whole-map reverse --
@pytest.mark.parametrize("m,n,q,reorth", [
    (12, 12, 0, True), (12, 12, 1, True), (12, 12, 2, True), (12, 12, 1, False),
    (12, 12, 2, False), (20, 14, 2, True), (17, 9, 1, False), (24, 24, 3, True),
])
def test_urv_backward_matches_finite_differences(m, n, q, reorth):
    A = _wellcond(1000 + m + 31 * n + q, m, n)
    G = oracle.gaussian(7, n, n)
    rng = np.random.default_rng(5 + q)
    Ubar = rng.standard_normal((m, n))
    Rbar = np.triu(rng.standard_normal((n, n)))
    Vbar = rng.standard_normal((n, n))

    def f(X):
        U, R, V = oracle.urv_g(X, G, q, reorth)
        return float(np.sum(Ubar * U) + np.sum(Rbar * R) + np.sum(Vbar * V))

    Abar = adjoint.urv_backward_g(A, G, q, reorth, Ubar, Rbar, Vbar)
    for t in range(3):
        D = rng.standard_normal((m, n))
        fd = _fd_directional(f, A, D, 1e-6)
        an = float(np.sum(Abar * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (t, fd, an)


def test_urv_backward_seeded_equals_explicit_g():
    A = _wellcond(3, 10, 10)
    rng = np.random.default_rng(1)
    Ub, Rb, Vb = rng.standard_normal((10, 10)), np.triu(rng.standard_normal((10, 10))), rng.standard_normal((10, 10))
    a = adjoint.urv_backward(A, 2, True, 11, Ub, Rb, Vb)
    b = adjoint.urv_backward_g(A, oracle.gaussian(11, 10, 10), 2, True, Ub, Rb, Vb)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("q,reorth", [(0, True), (1, True), (2, True), (2, False)])
def test_truncated_loss_full_rank_gradient_is_identity_gradient(q, reorth):
    # k = n: A_k = U R V^T = A exactly, so dL/dA = 2 (A - B) whatever G is.
    m, n = 16, 12
    A = _wellcond(77 + q, m, n)
    B = np.random.default_rng(9).standard_normal((m, n))
    G = oracle.gaussian(7, n, n)
    U, R, V = oracle.urv_g(A, G, q, reorth)
    L, Ub, Rb, Vb = adjoint.truncated_loss_cotangents(U, R, V, n, B)
    assert abs(L - np.sum((A - B) ** 2)) <= 1e-12 * L
    Abar = adjoint.urv_backward_g(A, G, q, reorth, Ub, Rb, Vb)
    ref = 2.0 * (A - B)
    assert np.linalg.norm(Abar - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("m,n,k,q,reorth", [
    (16, 16, 5, 0, True), (16, 16, 5, 1, True), (20, 16, 6, 2, True), (16, 16, 4, 2, False),
    (24, 18, 9, 1, False),
])
def test_truncated_loss_gradient_matches_projection_formula(m, n, k, q, reorth):
    A = _wellcond(300 + 7 * k + q, m, n, lo=0.5)
    B = np.random.default_rng(9).standard_normal((m, n))
    G = oracle.gaussian(7, n, n)
    U, R, V = oracle.urv_g(A, G, q, reorth)
    L, Ub, Rb, Vb = adjoint.truncated_loss_cotangents(U, R, V, k, B)
    Abar = adjoint.urv_backward_g(A, G, q, reorth, Ub, Rb, Vb)
    L2, Abar2 = adjoint.truncated_loss_grad_projection(A, G, q, k, B)
    assert abs(L - L2) <= 1e-11 * L
    assert np.linalg.norm(Abar - Abar2) <= 1e-8 * np.linalg.norm(Abar2)


def test_projection_formula_matches_finite_differences():
    m, n, k, q = 14, 12, 4, 2
    A = _wellcond(5, m, n, lo=0.5)
    B = np.random.default_rng(2).standard_normal((m, n))
    G = oracle.gaussian(3, n, n)
    _, Abar = adjoint.truncated_loss_grad_projection(A, G, q, k, B)
    rng = np.random.default_rng(4)
    f = lambda X: adjoint.truncated_loss_grad_projection(X, G, q, k, B)[0]
    for _ in range(3):
        D = rng.standard_normal((m, n))
        fd = _fd_directional(f, A, D, 1e-6)
        an = float(np.sum(Abar * D))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_q0_vbar_does_not_reach_abar():
    # q = 0: V = Q(G) is independent of A, so only (Ubar, Rbar) and the Vbar
    # that flows through C = A V matter; a change of Vbar alone changes nothing.
    m, n = 11, 8
    A = _wellcond(6, m, n)
    G = oracle.gaussian(5, n, n)
    rng = np.random.default_rng(0)
    Ub, Rb = rng.standard_normal((m, n)), np.triu(rng.standard_normal((n, n)))
    a = adjoint.urv_backward_g(A, G, 0, True, Ub, Rb, rng.standard_normal((n, n)))
    b = adjoint.urv_backward_g(A, G, 0, True, Ub, Rb, np.zeros((n, n)))
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
