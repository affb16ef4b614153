"""Pins for oracle.ridge: Eq. (1)-(3), (5) and the closed form against library routines and identities."""

import numpy as np
import pytest

from oracle import ridge
from paper_1602_02350_gb300 import synth


def _small(n=64, d=12, seed=5):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -1.5, 0.1, seed)
    return X.numpy(), y.numpy()


def test_cholesky_matches_lapack():
    A = synth.random_symmetric(20, 3) + 1e-3 * np.eye(20)
    L = ridge.cholesky(A)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        ridge.cholesky(-np.eye(3))


def test_closed_form_matches_library_solve_and_is_stationary():
    X, y = _small()
    lam = 1e-3
    w = ridge.closed_form(X, y, lam)
    n, d = X.shape
    ref = np.linalg.solve(X.T @ X / n + lam * np.eye(d), X.T @ y / n)
    np.testing.assert_allclose(w, ref, rtol=1e-10)
    # first-order condition of Eq. (1): X^T (X w - y)/n + lam w = 0
    g = X.T @ (X @ w - y) / n + lam * w
    assert np.linalg.norm(g) < 1e-13 * np.linalg.norm(X.T @ y / n)


def test_excess_identity_and_brute_force_minimum():
    X, y = _small(seed=9)
    lam = 1e-2
    ws = ridge.closed_form(X, y, lam)
    rng = np.random.default_rng(0)
    for _ in range(5):
        w = ws + rng.standard_normal(X.shape[1])
        direct = ridge.objective(X, y, lam, w) - ridge.objective(X, y, lam, ws)
        assert ridge.excess(X, lam, w, ws) == pytest.approx(direct, rel=1e-10)
        assert direct > 0
    # brute force: no random perturbation of w* lowers the objective
    L0 = ridge.objective(X, y, lam, ws)
    for _ in range(50):
        assert ridge.objective(X, y, lam, ws + 1e-3 * rng.standard_normal(X.shape[1])) >= L0


def test_objective_against_explicit_sum():
    X, y = _small(n=7, d=3)
    w = np.array([0.3, -1.0, 2.0])
    lam = 0.7
    s = sum(0.5 * (w @ X[i] - y[i]) ** 2 for i in range(7)) / 7 + 0.35 * (w @ w)
    assert ridge.objective(X, y, lam, w) == pytest.approx(s, rel=1e-14)


def test_correlation_and_condition_number():
    X, _ = _small(n=200, d=8)
    C = ridge.correlation(X)
    np.testing.assert_allclose(C, sum(np.outer(x, x) for x in X) / 200, rtol=1e-12)
    lam = 1e-2
    ev = np.linalg.eigvalsh(C)
    expect = np.sum(ev + lam) / (ev[0] + lam)          # Eq. (3), right-hand form
    assert ridge.avg_condition_number(C + lam * np.eye(8)) == pytest.approx(expect, rel=1e-12)
    # whitening: P = C + lam I gives kappa^ = d exactly (Sec. 1)
    H = C + lam * np.eye(8)
    e, U = np.linalg.eigh(H)
    Pm = (U / np.sqrt(e)) @ U.T
    assert ridge.avg_condition_number(Pm @ H @ Pm) == pytest.approx(8.0, rel=1e-10)


def test_speedup_ratio_special_cases():
    # flat spectrum: no gain; k = d: sum / (d lambda_d)
    assert ridge.speedup_ratio(np.ones(10), 3) == pytest.approx(1.0)
    ev = np.array([4.0, 2.0, 1.0, 0.5])
    assert ridge.speedup_ratio(ev, 4) == pytest.approx(7.5 / 2.0)
    assert ridge.speedup_ratio(ev, 1) == pytest.approx(1.0)
    assert ridge.speedup_ratio(ev, 2) == pytest.approx(7.5 / (2 * 2.0 + 1.5))


def test_sketched_ratio_equals_the_spectral_ratio_with_exact_eigenvalues():
    """With sigma2 = the eigenvalues of C (what a perfect sketch returns) and tr(C) = ||X||_F^2 / n,
    the sketched form equals the ratio on the spectrum (Eq. after Thm 1) for every k."""
    X, _ = _small(n=200, d=30, seed=4)
    ev = np.sort(np.linalg.eigvalsh(ridge.correlation(X)))[::-1]
    trc = float((X * X).sum() / X.shape[0])
    for k in range(1, 31):
        assert ridge.speedup_ratio_sketched(ev, trc, k) == pytest.approx(ridge.speedup_ratio(ev, k), rel=1e-10)


def test_sketched_ratio_two_level_closed_form():
    """r eigenvalues a and d - r eigenvalues b < a: ratio(k) = T / (k a + (r - k) a + (d - r) b) = 1 for
    k <= r, and T / (d b) for k > r, with T = r a + (d - r) b; a dropped tail or a wrong k factor fails."""
    r, d, a, b = 5, 40, 3.0, 0.25
    ev = np.array([a] * r + [b] * (d - r))
    T = r * a + (d - r) * b
    for k in range(1, r + 1):
        assert ridge.speedup_ratio_sketched(ev, T, k) == pytest.approx(1.0, rel=1e-14)
    for k in range(r + 1, d + 1):
        assert ridge.speedup_ratio_sketched(ev, T, k) == pytest.approx(T / (d * b), rel=1e-14)
    # an underestimated head (a sketch that misses mass) moves it into the tail: the ratio drops
    assert ridge.speedup_ratio_sketched(0.5 * ev, T, r + 1) < T / (d * b)


def test_chunked_normal_equations_match_the_one_block_forms():
    """Block accumulation of X^T X, X^T y, y^T y (any split) and the quantities derived from them equal
    the direct forms: closed form, excess identity and objective."""
    X, y = _small(n=300, d=17, seed=12)
    lam = 3e-3
    blocks = [(X[:7], y[:7]), (X[7:150], y[7:150]), (X[150:], y[150:])]
    G, b, yy, n = ridge.normal_equations(blocks)
    assert n == 300
    np.testing.assert_allclose(G, ridge.correlation(X) * n, rtol=1e-12)
    np.testing.assert_allclose(b, X.T @ y, rtol=1e-12)
    assert yy == pytest.approx(float(y @ y), rel=1e-13)
    ws = ridge.closed_form_from_normal(G, b, n, lam)
    np.testing.assert_allclose(ws, ridge.closed_form(X, y, lam), rtol=1e-9)
    w = ws + 0.01 * np.arange(17)
    assert ridge.excess_from_normal(G, lam, n, w - ws) == pytest.approx(ridge.excess(X, lam, w, ws), rel=1e-10)
    assert ridge.objective_from_normal(G, b, yy, n, lam, w) == pytest.approx(ridge.objective(X, y, lam, w), rel=1e-10)
