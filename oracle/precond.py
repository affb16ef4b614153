"""Sketched preconditioner (Eq. (11)) and the preconditioned n+d components (Sec. 5.1, Alg. 3),
float64 (oracle; test infrastructure).

Scaling convention.  Eq. (11) is P^{-1/2} = c M with c = (sigma~_k^2 + lam)^{-1/2}
and M = I - V (I - D') V^T, D'_i = sqrt((sigma~_k^2 + lam) / (sigma~_i^2 + lam)).
The library (and this oracle) preconditions with M and drops c: the problem
min_w~ L(M w~) is Eq. (4) in the coordinates c w~, so w = M w~ minimises Eq. (1)
exactly and c is absorbed by the step size, which is set from the smoothness
constants of the M-scaled components.
"""

import numpy as np


def dprime(sigma2, lam):
    """D'_i = sqrt((sigma~_k^2 + lam) / (sigma~_i^2 + lam)); D'_k = 1, all D'_i <= 1."""
    s = np.asarray(sigma2, np.float64)
    return np.sqrt((s[-1] + lam) / (s + lam))


def p_inv_sqrt(V, sigma2, lam):
    """Eq. (11): sum_i u_i u_i^T / sqrt(sigma_i^2 + lam) + (I - sum_i u_i u_i^T) / sqrt(sigma_k^2 + lam)."""
    V = np.asarray(V, np.float64)
    s = np.asarray(sigma2, np.float64)
    d = V.shape[0]
    proj = V @ V.T
    return (V / np.sqrt(s + lam)) @ V.T + (np.eye(d) - proj) / np.sqrt(s[-1] + lam)


def scale_c(sigma2, lam):
    """c = (sigma~_k^2 + lam)^{-1/2}, the factor Eq. (11) puts on the non-leading directions."""
    return 1.0 / np.sqrt(float(np.asarray(sigma2)[-1]) + lam)


def m_matrix(V, sigma2, lam):
    """M = P^{-1/2} / c (Eq. (11) without its scalar)."""
    return p_inv_sqrt(V, sigma2, lam) / scale_c(sigma2, lam)


def transform(X, M):
    """x~_i = M x_i for the n examples (rows of X M, M symmetric) and b_j = M e_j
    (rows of M): the data transform of Alg. 3 and the regulariser vectors of Sec. 5.1."""
    X = np.asarray(X, np.float64)
    M = np.asarray(M, np.float64)
    return X @ M, M.copy()


def components(Xt, B, y, lam):
    """The N = n + d components of Sec. 5.1 written as rows z_i with weights gamma_i:

        l~_i(w)     = gamma_i 1/2 (w^T z_i - y_i)^2,
        z_i = x~_i, gamma_i = (n+d)/n,       y_i as given     (i <= n)
        z_i = b_j,  gamma_i = lam (n+d),     y_i = 0          (i = n + j)

    so that L~(w) = (1/N) sum_i l~_i(w).  The regulariser components keep the 1/2
    of Sec. 5.1 (Alg. 3 prints them without it).
    """
    Xt = np.asarray(Xt, np.float64)
    n, d = Xt.shape
    N = n + d
    Z = np.vstack([Xt, np.asarray(B, np.float64)])
    yz = np.concatenate([np.asarray(y, np.float64), np.zeros(d)])
    gamma = np.concatenate([np.full(n, N / n), np.full(d, lam * N)])
    return Z, yz, gamma


def smoothness(Z, gamma):
    """beta_i = gamma_i ||z_i||^2 (Alg. 3: ((n+d)/n)||x~_i||^2 and lam(n+d)||b_j||^2; the
    printed ||b_i|| is read as squared, which is the Hessian norm of l~_{n+j})."""
    Z = np.asarray(Z, np.float64)
    return np.asarray(gamma) * np.einsum("ij,ij->i", Z, Z)


def beta_hat(beta):
    """beta^ = (1/N) sum_i beta_i (Eq. (8); the 1/n printed in Alg. 3 is read as 1/(n+d),
    as in the proof of Thm 4)."""
    return float(np.mean(np.asarray(beta, np.float64)))


def theory_defaults(beta, lam):
    """Thm 2 parameters: eta = 0.1 / beta^, m = ceil(kappa^_F) with kappa^_F = beta^ / alpha and
    the strong-convexity constant alpha taken as lam (parity unpinned: a heuristic
    lower bound, exact for the exact sketched preconditioner up to (sigma~_k^2+lam)/(lambda_k+lam))."""
    bh = beta_hat(beta)
    return 0.1 / bh, int(np.ceil(bh / lam))
