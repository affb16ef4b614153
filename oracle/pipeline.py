"""Sketched Preconditioned SVRG end to end (Alg. 3), float64 (oracle; test infrastructure)."""

import numpy as np

from . import precond, ridge, sketch, svrg


def scsvrg(X, y, lam, k, sketch_seed, svrg_seed, epochs, eta=None, m=None,
           kind="gaussian", s=0, q=1, uniform=False, average=True, history=False, eta_mult=None):
    """Alg. 3: sketch (Alg. 2) -> preconditioner (Eq. (11)) -> transformed data and
    regulariser vectors (Sec. 5.1) -> smoothness beta_i -> SVRG (Alg. 1) -> w = M w~.

    ``eta`` / ``m`` default to the Thm 2 values (``precond.theory_defaults``);
    ``eta_mult`` sets eta = eta_mult / beta^ instead (the paper tunes eta, Sec. 6).
    Returns a dict with the solution in original coordinates and the
    intermediate objects; with ``history`` also every epoch's snapshot mapped
    back to original coordinates.
    """
    X = np.asarray(X, np.float64)
    V, sigma2 = sketch.block_lanczos(X, k, sketch_seed, q=q, kind=kind, s=s)
    M = precond.m_matrix(V, sigma2, lam)
    Xt, B = precond.transform(X, M)
    Z, yz, gamma = precond.components(Xt, B, y, lam)
    beta = precond.smoothness(Z, gamma)
    eta_d, m_d = precond.theory_defaults(beta, lam)
    if eta is None:
        eta = eta_d if eta_mult is None else eta_mult / precond.beta_hat(beta)
    m = m_d if m is None else m
    snaps = svrg.solve(Z, yz, gamma, beta, eta, m, epochs, svrg_seed, uniform=uniform, average=average)
    out = {"w": M @ snaps[-1], "w_tilde": snaps[-1], "V": V, "sigma2": sigma2, "M": M,
           "beta": beta, "eta": eta, "m": m}
    if history:
        out["history"] = [M @ w for w in snaps]
    return out


def plain_svrg(X, y, lam, svrg_seed, epochs, eta=None, m=None, uniform=False):
    """Unpreconditioned SVRG on the same n+d components (M = I), the k = 0 special case."""
    X = np.asarray(X, np.float64)
    d = X.shape[1]
    Z, yz, gamma = precond.components(X, np.eye(d), y, lam)
    beta = precond.smoothness(Z, gamma)
    eta_d, m_d = precond.theory_defaults(beta, lam)
    snaps = svrg.solve(Z, yz, gamma, beta, eta_d if eta is None else eta,
                       m_d if m is None else m, epochs, svrg_seed, uniform=uniform)
    return snaps


def relative_history(X, y, lam, ws):
    """Relative suboptimality of each w in ``ws`` against the closed form."""
    w_star = ridge.closed_form(X, y, lam)
    return [ridge.rel_suboptimality(X, y, lam, w, w_star) for w in ws]
