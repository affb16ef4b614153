"""Pins for oracle.svrg and oracle.pipeline (Alg. 1, Alg. 3): chain rule and finite differences,
unbiasedness by enumeration, convergence to the Cholesky closed form, k = 0 reduction, resume."""

import numpy as np
import pytest

from oracle import pipeline, precond, ridge, sketch, streams, svrg
from paper_1602_02350_gb300 import synth


def _setup(n=120, d=10, lam=1e-2, k=3, seed=4):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -1.5, 0.1, seed)
    X, y = X.numpy(), y.numpy()
    V, s2 = sketch.block_lanczos(X, k, seed=seed + 1)
    M = precond.m_matrix(V, s2, lam)
    Z, yz, g = precond.components(*precond.transform(X, M), y, lam)
    return X, y, lam, M, Z, yz, g


def test_full_gradient_chain_rule_and_finite_differences():
    X, y, lam, M, Z, yz, g = _setup()
    n, d = X.shape
    wt = synth.random_vector(d, 1)
    mu = svrg.full_gradient(Z, yz, g, wt)
    # chain rule on Eq. (1): grad_w~ L(M w~) = M^T (X^T (X M w~ - y)/n + lam M w~)
    w = M @ wt
    ref = M.T @ (X.T @ (X @ w - y) / n + lam * w)
    np.testing.assert_allclose(mu, ref, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(svrg.full_gradient_fast(Z, yz, g, wt), mu, rtol=1e-12, atol=1e-15)
    # central differences of L(M w~)
    h = 1e-5
    fd = np.array([(ridge.objective(X, y, lam, M @ (wt + h * e)) - ridge.objective(X, y, lam, M @ (wt - h * e))) / (2 * h)
                   for e in np.eye(d)])
    np.testing.assert_allclose(mu, fd, rtol=1e-6, atol=1e-9)


def test_variance_reduced_direction_is_unbiased():
    """sum_i q_i v(i) = grad F(w) for any w, w_bar (enumerating every i exactly)."""
    X, y, lam, M, Z, yz, g = _setup(n=30, d=6)
    N, d = Z.shape
    beta = precond.smoothness(Z, g)
    _, _, q = svrg.sampling_table(beta)
    w_bar = synth.random_vector(d, 2)
    w = synth.random_vector(d, 3)
    v_bar = svrg.full_gradient(Z, yz, g, w_bar)
    ev = sum(q[i] * ((svrg.grad_component(Z, yz, g, i, w) - svrg.grad_component(Z, yz, g, i, w_bar)) / (N * q[i]) + v_bar)
             for i in range(N))
    np.testing.assert_allclose(ev, svrg.full_gradient(Z, yz, g, w), rtol=1e-11, atol=1e-14)


def test_svrg_converges_to_closed_form():
    X, y, lam, M, Z, yz, g = _setup()
    beta = precond.smoothness(Z, g)
    eta = 0.3 / precond.beta_hat(beta)
    snaps = svrg.solve(Z, yz, g, beta, eta, 2 * X.shape[0], 25, seed=7)
    ws = ridge.closed_form(X, y, lam)
    rel = [ridge.rel_suboptimality(X, y, lam, M @ w, ws) for w in snaps]
    assert rel[-1] < 1e-12
    assert rel[-1] < rel[0] * 1e-6


def test_k0_reduces_to_plain_svrg_and_uniform_sampling_converges():
    X, y, _ = synth.problem(80, 8, np.arange(1, 9) ** -1.0, 0.1, 11)
    X, y = X.numpy(), y.numpy()
    lam = 1e-2
    ws = ridge.closed_form(X, y, lam)
    snaps = pipeline.plain_svrg(X, y, lam, 3, 60, m=160)
    assert ridge.rel_suboptimality(X, y, lam, snaps[-1], ws) < 1e-10
    Z, yz, g = precond.components(X, np.eye(8), y, lam)
    beta = precond.smoothness(Z, g)
    snaps_u = svrg.solve(Z, yz, g, beta, 0.25 / beta.max(), 160, 60, 3, uniform=True)
    assert ridge.rel_suboptimality(X, y, lam, snaps_u[-1], ws) < 1e-6


def test_resume_at_epoch_boundary_is_bit_identical():
    X, y, lam, M, Z, yz, g = _setup(n=60, d=6)
    beta = precond.smoothness(Z, g)
    eta = 0.1 / precond.beta_hat(beta)
    full = svrg.solve(Z, yz, g, beta, eta, 50, 4, seed=5)
    half = svrg.solve(Z, yz, g, beta, eta, 50, 2, seed=5)
    rest = svrg.solve(Z, yz, g, beta, eta, 50, 2, seed=5, w0=half[-1], epoch0=2)
    np.testing.assert_array_equal(full[-1], rest[-1])


def test_last_iterate_option_and_zero_step():
    X, y, lam, M, Z, yz, g = _setup(n=40, d=5)
    beta = precond.smoothness(Z, g)
    _, _, q = svrg.sampling_table(beta)
    idx = streams.sample_indices(streams.cumulative(streams.quantize_weights(beta)), 1, 0, 30)
    w_bar = synth.random_vector(5, 9)
    np.testing.assert_allclose(svrg.epoch(Z, yz, g, w_bar, idx, q, 0.0), w_bar, rtol=1e-14)
    last = svrg.epoch(Z, yz, g, w_bar, idx[:1], q, 0.01, average=False)
    avg = svrg.epoch(Z, yz, g, w_bar, idx[:1], q, 0.01, average=True)
    np.testing.assert_array_equal(last, avg)        # one step: average == last iterate


@pytest.mark.slow
def test_alg3_fp64_config_reaches_1e10():
    """Alg. 3 on the FP64 workload (n = 4096, d = 256, k = 16, m = 2n): the oracle itself
    converges to the Cholesky solution."""
    cfg = synth.CONFIGS["fp64_n4096_d256"]
    X, y, _ = synth.config_problem(cfg)
    X, y = X.numpy(), y.numpy()
    out = pipeline.scsvrg(X, y, cfg.lam, cfg.k, cfg.seed_sketch, cfg.seed_svrg, epochs=cfg.epochs,
                          m=cfg.m, eta_mult=cfg.eta_mult, history=True)
    rel = pipeline.relative_history(X, y, cfg.lam, out["history"])
    assert rel[-1] < 1e-10


def test_chunked_full_gradient_equals_the_one_block_form():
    from oracle import precond
    rng = np.random.default_rng(3)
    n, d, lam = 90, 13, 1e-2
    Z = rng.standard_normal((n + d, d))
    y = rng.standard_normal(n)
    _, yz, g = precond.components(Z[:n], Z[n:], y, lam)
    w = rng.standard_normal(d)
    cuts = [0, 5, 47, 95, n + d]
    blocks = [(Z[a:b], yz[a:b], g[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    np.testing.assert_allclose(svrg.full_gradient_chunked(blocks, n + d, w), svrg.full_gradient(Z, yz, g, w),
                               rtol=1e-12, atol=1e-14)
