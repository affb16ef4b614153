"""Pins for oracle.catalyst (accelerated SVRG around Alg. 1): the proximal problem's components and
their minimiser, the alpha / extrapolation recursion, the kappa = 0 reduction to plain SVRG, and
convergence to the ridge solution."""

import numpy as np
import pytest

from oracle import catalyst, precond, ridge, sketch, svrg
from paper_1602_02350_gb300 import synth


def _setup(n=300, d=24, lam=1e-3, k=4, seed=3):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -1.5, 0.1, seed)
    X, y = X.numpy(), y.numpy()
    V, s2 = sketch.block_lanczos(X, k, seed + 1)
    M = precond.m_matrix(V, s2, lam)
    Z, yz, g = precond.components(*precond.transform(X, M), y, lam)
    return X, y, M, Z, yz, g, precond.smoothness(Z, g)


def test_alpha_recursion_and_extrapolation():
    q = 0.01
    a = np.sqrt(q)
    for _ in range(50):
        b = catalyst.next_alpha(a, q)
        assert 0 < b < 1
        assert b * b == pytest.approx((1 - b) * a * a + q * b, rel=1e-13)
        assert catalyst.extrapolation(a, b) == pytest.approx(a * (1 - a) / (a * a + b), rel=1e-15)
        a = b
    # alpha_0 = sqrt(q) is a fixed point of the recursion (the strongly convex choice of Catalyst)
    assert catalyst.next_alpha(np.sqrt(q), q) == pytest.approx(np.sqrt(q), rel=1e-13)


def test_proximal_components_reproduce_the_proximal_objective():
    """(1/N) sum_i f_i over the proximal problem's components equals L(M w~) + kappa/2 ||M w~ - c||^2 up to
    a constant in w~: differences between two points agree (the objective of Eq. (1) plus the proximal
    term), and the gradient vanishes at the closed-form proximal minimiser."""
    X, y, M, Z, yz, g, beta = _setup()
    n, d = X.shape
    lam, kappa = 1e-3, 0.05
    c = synth.random_vector(d, 7)
    y2, g2 = catalyst.subproblem(Z, yz, g, n, lam, kappa, c)

    def F(wt):
        return np.mean(0.5 * g2 * (Z @ wt - y2) ** 2)

    def G(wt):
        w = M @ wt
        return ridge.objective(X, y, lam, w) + 0.5 * kappa * np.sum((w - c) ** 2)

    a, b = synth.random_vector(d, 8), synth.random_vector(d, 9)
    assert F(a) - F(b) == pytest.approx(G(a) - G(b), rel=1e-10)
    wp = catalyst.proximal_minimiser(X, y, lam, kappa, c)
    wt = np.linalg.solve(M, wp)
    assert np.linalg.norm(svrg.full_gradient(Z, y2, g2, wt)) < 1e-12 * np.linalg.norm(svrg.full_gradient(Z, y2, g2, 0 * wt))


def test_kappa_zero_is_plain_svrg():
    """q = 1, alpha = 1, b = 0: the outer iterates are the epochs of Alg. 1 run back to back."""
    X, y, M, Z, yz, g, beta = _setup()
    n = X.shape[0]
    xs = catalyst.solve(Z, yz, g, beta, M, n, 1e-3, 0.0, 3, 2, 600, 1.0, 11)
    snaps = svrg.solve(Z, yz, g, beta, 1.0 / precond.beta_hat(beta), 600, 6, 11)
    for t in range(3):
        np.testing.assert_allclose(xs[t], M @ snaps[2 * t + 1], rtol=1e-12, atol=1e-15)


def test_catalyst_converges_to_the_ridge_solution():
    X, y, M, Z, yz, g, beta = _setup(lam=1e-4)
    n, d = X.shape
    N = n + d
    lam = 1e-4
    kappa = precond.beta_hat(beta) / N - lam
    assert kappa > 0
    xs = catalyst.solve(Z, yz, g, beta, M, n, lam, kappa, 12, 2, n, 1.0, 5)
    ws = ridge.closed_form(X, y, lam)
    rel = [ridge.rel_suboptimality(X, y, lam, x, ws) for x in xs]
    assert rel[-1] < 1e-8, rel
    assert rel[-1] < 1e-6 * rel[0]
