"""Pins of the oracle's randomized SVD (Section 6, Eqs. (rsvd1)-(rsvd4)) against
facts that are not its own code: the G-prefix convention of the Lemma, exact
recovery of matrices of rank <= l, the singular values of Q Q^T A never exceed
those of A, the Lemma itself (the range of U_rsvd is the range of the first l
columns of PowerURV's U for the same G), and the sign convention."""
import numpy as np
import pytest

import oracle
from oracle import rsvd as orsvd


def _mat(m, n, sig, seed):
    rng = np.random.default_rng(seed)
    Uh, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vh, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Uh * sig) @ Vh.T


def test_g_rsvd_is_the_prefix_of_the_powerurv_draw():
    G = oracle.gaussian(7, 40, 40)
    assert np.array_equal(oracle.gaussian(7, 40, 12), G[:, :12])


@pytest.mark.parametrize("q,reorth", [(0, False), (1, False), (2, True)])
def test_exact_low_rank_is_recovered(q, reorth):
    m, n, r, l = 50, 30, 6, 8
    sig = np.zeros(n)
    sig[:r] = np.linspace(3.0, 1.0, r)
    A = _mat(m, n, sig, 3)
    U, s, V = orsvd.rsvd(A, l, q, 11, reorth)
    assert np.linalg.norm(A - (U * s) @ V.T) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(s[:r], sig[:r], rtol=1e-12, atol=0)
    assert np.all(s[r:] <= 1e-12 * s[0])


@pytest.mark.parametrize("q", [0, 1, 2])
def test_singular_values_interlace_and_factors_are_orthonormal(q):
    m, n, l = 60, 40, 10
    A = np.random.default_rng(q).standard_normal((m, n))
    U, s, V = orsvd.rsvd(A, l, q, 5)
    sa = np.linalg.svd(A, compute_uv=False)
    assert np.all(s <= sa[:l] * (1 + 1e-12))
    assert np.all(np.diff(s) <= 0)
    assert np.linalg.norm(U.T @ U - np.eye(l)) <= 1e-13 * l
    assert np.linalg.norm(V.T @ V - np.eye(l)) <= 1e-13 * l
    for j in range(l):
        assert U[int(np.argmax(np.abs(U[:, j]))), j] > 0


@pytest.mark.parametrize("q,reorth", [(1, True), (2, True), (2, False)])
def test_lemma_range_equals_powerurv_leading_columns(q, reorth):
    # Section 6, Lemma: with G_rsvd = G(:, 1:l), range(U_rsvd) = range(U(:, 1:l)).
    m, n, l = 80, 50, 12
    A = _mat(m, n, np.linspace(1.0, 0.2, n), 21)
    G = oracle.gaussian(7, n, n)
    U, _, _ = oracle.urv_g(A, G, q, reorth)
    Ur, _, _ = orsvd.rsvd_g(A, G[:, :l], q, reorth)
    P1 = U[:, :l] @ U[:, :l].T
    P2 = Ur @ Ur.T
    assert np.linalg.norm(P1 - P2, 2) <= 1e-10


def test_more_power_steps_do_not_hurt_on_a_decaying_spectrum():
    m, n, l = 120, 80, 10
    A = _mat(m, n, 0.8 ** np.arange(n), 4)
    err = []
    for q in (0, 1, 2):
        U, s, V = orsvd.rsvd(A, l, q, 9)
        err.append(np.linalg.norm(A - (U * s) @ V.T, 2))
    sa = np.linalg.svd(A, compute_uv=False)
    assert err[2] <= err[0] and err[2] <= 1.05 * sa[l]
