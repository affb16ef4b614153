"""Pins for oracle.precond: Eq. (4) invariance, Lemma 1 spectrum, Thm 4 trace identity,
whitening, Lemmas 2-4 as soft checks."""

import numpy as np
import pytest

from oracle import precond, ridge, sketch
from paper_1602_02350_gb300 import synth


def _data(n=300, d=16, alpha=1.5, seed=2, noise=0.1):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -alpha, noise, seed)
    return X.numpy(), y.numpy()


def _exact(X, k):
    C = ridge.correlation(X)
    ev, U = np.linalg.eigh(C)
    return ev[::-1], U[:, ::-1], C


def test_dprime_properties():
    s2 = np.array([3.0, 1.0, 0.2])
    Dp = precond.dprime(s2, 0.1)
    assert Dp[-1] == 1.0 and np.all(Dp <= 1.0) and np.all(np.diff(Dp) >= 0)


def test_m_is_eq11_without_its_scalar_and_has_low_rank_form():
    V = synth.random_orthonormal(10, 3, 1)
    s2 = np.array([2.0, 0.5, 0.1])
    lam = 1e-2
    P = precond.p_inv_sqrt(V, s2, lam)
    np.testing.assert_allclose(P, P.T, atol=1e-15)
    M = precond.m_matrix(V, s2, lam)
    # M = I - V (I - D') V^T
    Dp = precond.dprime(s2, lam)
    np.testing.assert_allclose(M, np.eye(10) - (V * (1 - Dp)) @ V.T, atol=1e-14)
    # eigenvalues of P^{-1/2}: 1/sqrt(s2_i + lam) on V and 1/sqrt(s2_k + lam) elsewhere
    ev = np.sort(np.linalg.eigvalsh(P))
    expect = np.sort(np.concatenate([1 / np.sqrt(s2 + lam), np.full(7, 1 / np.sqrt(s2[-1] + lam))]))
    np.testing.assert_allclose(ev, expect, rtol=1e-12)


def test_whitening_gives_kappa_equal_d():
    """Sec. 1 / Thm 4: P = C + lam I (k = d, exact eigenpairs) gives kappa~ = d."""
    X, _ = _data(d=12)
    lam = 1e-3
    ev, U, C = _exact(X, 12)
    P = precond.p_inv_sqrt(U, ev, lam)
    H = P @ (C + lam * np.eye(12)) @ P
    np.testing.assert_allclose(H, np.eye(12), atol=1e-10)
    assert ridge.avg_condition_number(H) == pytest.approx(12.0, rel=1e-9)


def test_lemma1_spectrum_and_bound():
    X, _ = _data(d=20, alpha=1.2)
    lam, k = 1e-3, 5
    ev, U, C = _exact(X, k)
    P = precond.p_inv_sqrt(U[:, :k], ev[:k], lam)
    H = P @ (C + lam * np.eye(20)) @ P
    got = np.sort(np.linalg.eigvalsh(H))
    expect = np.sort(np.concatenate([np.ones(k), (ev[k:] + lam) / (ev[k - 1] + lam)]))
    np.testing.assert_allclose(got, expect, rtol=1e-9)
    bound = (k * ev[k - 1] + ev[k:].sum()) / lam + 20          # Eq. (10)
    assert ridge.avg_condition_number(H) <= bound


def test_components_reproduce_eq1_invariance_and_hessian():
    """L~(w~) = (1/N) sum_i l~_i(w~) equals L(M w~) (Eq. (4) with P^{-1/2} -> M) and the
    Hessian of L~ is M (C + lam I) M (proof of Thm 4)."""
    X, y = _data()
    n, d = X.shape
    lam = 1e-2
    V, s2 = sketch.block_lanczos(X, 4, seed=5)
    M = precond.m_matrix(V, s2, lam)
    Xt, B = precond.transform(X, M)
    Z, yz, g = precond.components(Xt, B, y, lam)
    rng = np.random.default_rng(3)
    for _ in range(4):
        wt = rng.standard_normal(d)
        Lt = np.mean(g * 0.5 * (Z @ wt - yz) ** 2)
        assert Lt == pytest.approx(ridge.objective(X, y, lam, M @ wt), rel=1e-12)
    Hs = (Z * g[:, None]).T @ Z / (n + d)
    np.testing.assert_allclose(Hs, M @ (ridge.correlation(X) + lam * np.eye(d)) @ M, rtol=1e-10, atol=1e-14)


def test_thm4_average_smoothness_equals_trace():
    X, y = _data(n=500, d=24)
    lam = 1e-3
    V, s2 = sketch.block_lanczos(X, 6, seed=1)
    M = precond.m_matrix(V, s2, lam)
    Z, yz, g = precond.components(*precond.transform(X, M), y, lam)
    beta = precond.smoothness(Z, g)
    tr = np.trace(M @ (ridge.correlation(X) + lam * np.eye(24)) @ M)
    assert precond.beta_hat(beta) == pytest.approx(tr, rel=1e-12)
    # each beta_i is the spectral norm of the rank-one Hessian of l~_i
    i = 7
    assert beta[i] == pytest.approx(np.linalg.norm(g[i] * np.outer(Z[i], Z[i]), 2), rel=1e-12)


def test_sketched_preconditioner_lemmas_soft():
    """Lemmas 2-4 (Thm 5) hold under the Thm 3 event; with q = Theta(log n) Block Lanczos
    that event has probability >= 9/10.  In the c-free scaling the bounds carry c^2."""
    X, _ = _data(n=800, d=40, alpha=1.5, seed=6)
    lam, k = 1e-4, 6
    C = ridge.correlation(X)
    ev = np.sort(np.linalg.eigvalsh(C))[::-1]
    ok = 0
    for seed in range(10):
        V, s2 = sketch.block_lanczos(X, k, seed=seed, q=6)
        P = precond.p_inv_sqrt(V, s2, lam)
        H = P @ (C + lam * np.eye(40)) @ P
        e = np.sort(np.linalg.eigvalsh(H))[::-1]
        c1 = e[0] <= 17
        c2 = np.all(e[k:] <= 2 * (ev[k:] + lam) / (ev[k - 1] + lam) * (1 + 1e-9))
        # Lemma 4, read with C + lam I as in its proof
        c4 = e[-1] >= lam / (19 * (ev[k - 1] + lam))
        ok += bool(c1 and c2 and c4)
    assert ok >= 9


def test_theory_defaults():
    beta = np.array([1.0, 3.0])
    eta, m = precond.theory_defaults(beta, 0.5)
    assert eta == pytest.approx(0.05) and m == 4
