"""Accelerated SVRG by Catalyst (Lin, Mairal and Harchaoui, NIPS 2015), the acceleration the paper
invokes in Sec. 1 and in Thm 1 ("or ... if we use accelerated SVRG"), around the oracle's SVRG on
the preconditioned components, float64 (oracle; test infrastructure).

Outer iteration t minimises the proximal problem
    G_t(w) = L(w) + (kappa/2) ||w - c_{t-1}||^2,
a ridge problem with regularisation lam + kappa centred at c' = kappa c / (lam + kappa) (up to a
constant).  In the n + d component form of Sec. 5.1 (w = M w~, regulariser rows b_j = M e_j) only
the regulariser rows change: their weight becomes (lam + kappa)(n + d) and their label c'_j,
because (M e_j)^T w~ = w_j.
The inner solver is Alg. 1 warm-started at the previous outer iterate; then
    alpha_t^2 = (1 - alpha_t) alpha_{t-1}^2 + q alpha_t,  q = lam / (lam + kappa),
    b_t = alpha_{t-1} (1 - alpha_{t-1}) / (alpha_{t-1}^2 + alpha_t),
    c_t = x_t + b_t (x_t - x_{t-1}),
with alpha_0 = sqrt(q) (the strongly convex choice of Catalyst).
"""

import numpy as np

from . import precond, svrg


def next_alpha(alpha_prev, q):
    """The positive root of a^2 = (1 - a) alpha_prev^2 + q a."""
    b = alpha_prev * alpha_prev - q
    return 0.5 * (-b + np.sqrt(b * b + 4.0 * alpha_prev * alpha_prev))


def extrapolation(alpha_prev, alpha):
    """b_t = alpha_{t-1} (1 - alpha_{t-1}) / (alpha_{t-1}^2 + alpha_t)."""
    return alpha_prev * (1.0 - alpha_prev) / (alpha_prev * alpha_prev + alpha)


def subproblem(Z, yz, gamma, n, lam, kappa, center):
    """Labels and weights of the proximal problem's components: rows i < n unchanged, regulariser
    rows weighted (lam + kappa)(n + d) with labels kappa c_j / (lam + kappa)."""
    N, d = Z.shape
    y2 = np.array(yz, np.float64)
    g2 = np.array(gamma, np.float64)
    y2[n:] = kappa / (lam + kappa) * np.asarray(center, np.float64)
    g2[n:] = (lam + kappa) * N
    return y2, g2


def solve(Z, yz, gamma, beta, M, n, lam, kappa, outer, epochs, m, eta_mult, seed, beta_scale=None):
    """Catalyst with ``outer`` iterations of ``epochs`` epochs of Alg. 1 each (m steps, eta = eta_mult /
    beta^ of the proximal problem's smoothness constants, epoch numbers continuing across the outer
    iterations).  ``beta`` are the smoothness constants of the original components; those of the
    proximal problem are beta with the regulariser rows scaled by (lam + kappa) / lam (the weight
    changes, the rows do not).  Returns the outer iterates x_t (original coordinates)."""
    N, d = Z.shape
    q = lam / (lam + kappa)
    scale = (lam + kappa) / lam if beta_scale is None else beta_scale
    beta2 = np.array(beta, np.float64)
    beta2[n:] = beta2[n:] * scale
    eta = eta_mult / precond.beta_hat(beta2)
    alpha = np.sqrt(q)
    wt = np.zeros(d)                     # preconditioned iterate (warm start)
    x_prev = M @ wt
    c = x_prev.copy()
    xs = []
    for t in range(outer):
        y2, g2 = subproblem(Z, yz, gamma, n, lam, kappa, c)
        snaps = svrg.solve(Z, y2, g2, beta2, eta, m, epochs, seed, w0=wt, epoch0=t * epochs)
        wt = snaps[-1]
        x = M @ wt
        a_new = next_alpha(alpha, q)
        c = x + extrapolation(alpha, a_new) * (x - x_prev)
        alpha, x_prev = a_new, x
        xs.append(x)
    return xs


def proximal_minimiser(X, y, lam, kappa, center):
    """Closed form of min_w L(w) + (kappa/2)||w - c||^2: (C + (lam + kappa) I) w = X^T y / n + kappa c."""
    X = np.asarray(X, np.float64)
    n, d = X.shape
    A = X.T @ X / n + (lam + kappa) * np.eye(d)
    return np.linalg.solve(A, X.T @ np.asarray(y, np.float64) / n + kappa * np.asarray(center, np.float64))
