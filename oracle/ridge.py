"""Ridge-regression objective and its closed form, float64 (oracle; test infrastructure).

Rows of ``X`` are the examples x_i (n x d, row-major); the paper's d x n matrix
whose i-th column is x_i (Sec. 5.3) is the same memory read transposed.
"""

import numpy as np


def objective(X, y, lam, w):
    """L(w) = (1/n) sum_i 1/2 (w^T x_i - y_i)^2 + (lam/2) ||w||^2  -- Eq. (1)."""
    X = np.asarray(X, np.float64)
    r = X @ np.asarray(w, np.float64) - np.asarray(y, np.float64)
    return 0.5 * float(r @ r) / X.shape[0] + 0.5 * lam * float(np.dot(w, w))


def correlation(X):
    """C = (1/n) sum_i x_i x_i^T  -- Eq. (2)."""
    X = np.asarray(X, np.float64)
    return X.T @ X / X.shape[0]


def avg_condition_number(H):
    """kappa_hat(H) = tr(H) / lambda_d(H) for a symmetric positive definite H -- Eq. (3).

    For H = C + lam I this is sum_i (lambda_i + lam) / (lambda_d + lam).
    """
    ev = np.linalg.eigvalsh(np.asarray(H, np.float64))
    return float(np.trace(H) / ev[0])


def cholesky(A):
    """Lower-triangular L with L L^T = A, by the textbook column (Cholesky-Banachiewicz) order."""
    A = np.asarray(A, np.float64)
    d = A.shape[0]
    L = np.zeros_like(A)
    for j in range(d):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if s <= 0.0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def closed_form(X, y, lam):
    """w* solving (C + lam I) w = (1/n) sum_i y_i x_i (Sec. 3), via our own Cholesky."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    A = correlation(X) + lam * np.eye(d)
    b = X.T @ np.asarray(y, np.float64) / n
    L = cholesky(A)
    # forward then backward substitution
    z = np.zeros(d)
    for i in range(d):
        z[i] = (b[i] - L[i, :i] @ z[:i]) / L[i, i]
    w = np.zeros(d)
    for i in range(d - 1, -1, -1):
        w[i] = (z[i] - L[i + 1:, i] @ w[i + 1:]) / L[i, i]
    return w


def excess(X, lam, w, w_star):
    """L(w) - L(w*) = 1/2 e^T (C + lam I) e with e = w - w*, exact for a quadratic
    with gradient zero at w*; written as (1/2n)||X e||^2 + (lam/2)||e||^2 so that no
    cancellation between two nearly equal objective values occurs."""
    X = np.asarray(X, np.float64)
    e = np.asarray(w, np.float64) - np.asarray(w_star, np.float64)
    Xe = X @ e
    return 0.5 * float(Xe @ Xe) / X.shape[0] + 0.5 * lam * float(e @ e)


def rel_suboptimality(X, y, lam, w, w_star):
    """(L(w) - L(w*)) / L(w*), the accuracy measure the solver is judged by."""
    return excess(X, lam, w, w_star) / objective(X, y, lam, w_star)


def speedup_ratio(eigs, k):
    """Eq. (5): sum_i lambda_i / (k lambda_k + sum_{i>k} lambda_i), eigenvalues descending."""
    ev = np.sort(np.asarray(eigs, np.float64))[::-1]
    return float(ev.sum() / (k * ev[k - 1] + ev[k:].sum()))


def speedup_ratio_sketched(sigma2, trace_c, k):
    """The same ratio (after Thm 1) from a sketch: sum_i lambda_i = tr(C), lambda_i ~ sigma2[i-1] for
    i <= k, and the tail sum_{i>k} lambda_i = tr(C) - sum_{i<=k} sigma2[i-1].  With exact eigenvalues
    (sigma2 = the spectrum of C) this is ``speedup_ratio``."""
    s = np.asarray(sigma2, np.float64)
    head = float(np.sum(s[:k]))
    return float(trace_c / (k * s[k - 1] + (trace_c - head)))


def normal_equations(chunks):
    """(X^T X, X^T y, y^T y, n) accumulated in float64 over row blocks (X_b, y_b) given in order, for
    data too large to hold in float64 at once; each block is converted to float64 before its
    products.  With one block this is correlation(X) * n and X^T y."""
    G = b = None
    yy, n = 0.0, 0
    for Xb, yb in chunks:
        Xb = np.asarray(Xb, np.float64)
        yb = np.asarray(yb, np.float64)
        if G is None:
            G = np.zeros((Xb.shape[1], Xb.shape[1]))
            b = np.zeros(Xb.shape[1])
        G += Xb.T @ Xb
        b += Xb.T @ yb
        yy += float(yb @ yb)
        n += Xb.shape[0]
    return G, b, yy, n


def closed_form_from_normal(G, b, n, lam):
    """w* of Eq. (1) from X^T X and X^T y: (G/n + lam I) w = b/n by a Cholesky factorisation and two
    triangular solves (the steps of ``closed_form``; LAPACK's factorisation, since d may be thousands)."""
    import scipy.linalg as sla
    d = G.shape[0]
    A = G / n + lam * np.eye(d)
    L = np.linalg.cholesky(A)
    z = sla.solve_triangular(L, b / n, lower=True)
    return sla.solve_triangular(L.T, z, lower=False)


def excess_from_normal(G, lam, n, e):
    """1/2 e^T (C + lam I) e with C = G / n (the excess of Eq. (1) at w* + e, as ``excess``)."""
    e = np.asarray(e, np.float64)
    return 0.5 * float(e @ (G @ e)) / n + 0.5 * lam * float(e @ e)


def objective_from_normal(G, b, yy, n, lam, w):
    """L(w) of Eq. (1) expanded through the normal equations: (w^T G w - 2 b^T w + y^T y)/(2n) + lam/2 ||w||^2."""
    w = np.asarray(w, np.float64)
    return (float(w @ (G @ w)) - 2.0 * float(b @ w) + yy) / (2.0 * n) + 0.5 * lam * float(w @ w)
