"""The quantities plotted in the paper's quality experiments, computed from a
factorization in FP64 with numpy (shared by the oracle and the GPU tests).

Figure 3 (Section 3): how well R reveals the rank, sigma_k(R11) against
sigma_k(A) and sigma_1(R22) against sigma_{k+1}(A), for k = 1..n-1.
Figures 5-7 (Section 7): the rank-k approximation error ||A - U(:,1:k) R(1:k,:) V^T||_2,
equal to sigma_1(R22) because R is upper triangular, against the optimum sigma_{k+1}(A).
Figures 9-10 (Section 6, the Lemma): ||A - U_k U_k^T A||_2 for PowerURV's U and
the RSVD's U_rsvd (l = 60), equal at k = l.
"""
import numpy as np

# columns whose optimal error sigma_{k+1} is above rounding
RELEVANT = 1e-12


def rank_revealing(A, R):
    """(sigma(A), sigma_k(R11) for k = 1..n-1, sigma_1(R22) for k = 1..n-1, mask of relevant k)."""
    n = A.shape[1]
    sa = np.linalg.svd(A, compute_uv=False)
    r11 = np.array([np.linalg.svd(R[:k, :k], compute_uv=False)[-1] for k in range(1, n)])
    r22 = np.array([np.linalg.norm(R[k:, k:], 2) for k in range(1, n)])
    mask = sa[1:] > RELEVANT * sa[0]
    return sa, r11, r22, mask


def approx_errors(A, U, R, V, ks):
    """||A - U(:,1:k) R(1:k,:) V^T||_2 for k in ks."""
    return np.array([np.linalg.norm(A - U[:, :k] @ R[:k, :] @ V.T, 2) for k in ks])


def projection_errors(A, Q, ks):
    """||A - Q(:,1:k) Q(:,1:k)^T A||_2 for k in ks."""
    return np.array([np.linalg.norm(A - Q[:, :k] @ (Q[:, :k].T @ A), 2) for k in ks])


def row_projection_errors(A, V, ks):
    """||A - A V(:,1:k) V(:,1:k)^T||_2 for k in ks."""
    return np.array([np.linalg.norm(A - (A @ V[:, :k]) @ V[:, :k].T, 2) for k in ks])


def check_quality(name, A, facts):
    """The claims of Figures 3 and 5-7 on one matrix.  `facts` maps q to (U, R, V).
    Returns a row of the summary table per q."""
    rows = []
    med = {}
    for q, (U, R, V) in facts.items():
        sa, r11, r22, mask = rank_revealing(A, R)
        # interlacing: exact invariants of any orthogonal U, V and triangular R (up to rounding)
        assert np.all(r11[mask] <= sa[:-1][mask] * (1 + 1e-10)), (name, q)
        assert np.all(r22[mask] >= sa[1:][mask] * (1 - 1e-10)), (name, q)
        ks = np.arange(1, A.shape[1])
        e = approx_errors(A, U, R, V, ks)
        assert np.allclose(e, r22, rtol=1e-10, atol=1e-14 * sa[0])
        ratio = e[mask] / sa[1:][mask]
        med[q] = float(np.median(ratio))
        rows.append((name, q, med[q], float(ratio.max()), float(np.median(r11[mask] / sa[:-1][mask]))))
    # q >= 1 track the optimum closely; without power steps the errors are several times larger
    assert med[1] <= 1.5 and med[2] <= 1.5, (name, med)
    assert med[2] <= med[1] * 1.05 and med[1] <= med[0], (name, med)
    assert med[0] >= 1.5 * med[2], (name, med)
    return rows


def check_lemma(A, Upurv, Vpurv, Ursvd, Vrsvd, ell):
    """Figures 9-10: equal errors at k = l; RSVD's extra application of A gives the better
    leading columns (U and V) for k well below l."""
    ks = np.arange(1, ell + 1)
    eu, er = projection_errors(A, Upurv, ks), projection_errors(A, Ursvd, ks)
    assert abs(eu[-1] - er[-1]) <= 1e-10 * er[-1]
    assert np.median(eu[: ell // 2] / er[: ell // 2]) > 1.0
    ev, evr = row_projection_errors(A, Vpurv, ks), row_projection_errors(A, Vrsvd, ks)
    assert np.median(ev[: ell // 2] / evr[: ell // 2]) > 1.0
    return (float(eu[-1]), float(er[-1]), float(np.median(eu[: ell // 2] / er[: ell // 2])),
            float(np.median(ev[: ell // 2] / evr[: ell // 2])))
