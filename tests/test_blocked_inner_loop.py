"""The blocked form of Alg. 1's inner loop that the CUDA kernels run, checked against the oracle's
step-by-step loop on the CPU (float64).  Per block of B sampled components z_0..z_{B-1}, starting
from delta_0 = w - w_bar, with p_j = z_j^T delta_0, h_j = z_j^T mu, G the block's Gram matrix, L
its strictly lower part and K = diag(kappa_j), kappa_j = gamma_{i_j} / (N q_{i_j}):

    a = R (p - eta (j . h)),   R = (I + eta K L)^{-1} K      (a_j = kappa_j z_j^T delta_j)
    delta_B = delta_0 - eta (B mu + sum_j a_j z_j)
    sum_{t=1..B} delta_t = B delta_0 - eta (B (B + 1) / 2 mu + sum_j (B - j) a_j z_j)

which is exact algebra: every iterate of the sequential loop is represented.  R is formed by
forward substitution column by column, and c = -eta R (j . h) by the same substitution with the
right-hand side kappa . j . h, as the preparation kernels do."""

import numpy as np
import pytest

from oracle import svrg


def _forward_subst(G, kap, eta, rhs):
    """r_l = kap_l (rhs_l - eta sum_{l' < l} G[l][l'] r_l')."""
    B = len(kap)
    r = np.zeros(B)
    for l in range(B):
        r[l] = kap[l] * (rhs[l] - eta * G[l, :l] @ r[:l])
    return r


def _blocked_epoch(Z, gamma, w_bar, idx, inv_nq, eta, mu, B, average):
    m = len(idx)
    delta = np.zeros(Z.shape[1])
    run = np.zeros(Z.shape[1])
    for b0 in range(0, m, B):
        rows = np.asarray(idx[b0:b0 + B])
        Bb = len(rows)
        Zb = Z[rows]
        kap = gamma[rows] * inv_nq[b0:b0 + Bb]
        G = Zb @ Zb.T
        p = Zb @ delta
        h = Zb @ mu
        jv = np.arange(Bb, dtype=np.float64)
        # R column by column (rhs = e_c), then a = R p + c with c = -eta R (j . h)
        R = np.stack([_forward_subst(G, kap, eta, np.eye(Bb)[c]) for c in range(Bb)], axis=1)
        c = -eta * _forward_subst(G, kap, eta, jv * h)
        a = R @ p + c
        run += Bb * delta - eta * (Bb * (Bb + 1) / 2 * mu + ((Bb - jv) * a) @ Zb)
        delta = delta - eta * (Bb * mu + a @ Zb)
    return w_bar + (run / m if average else delta)


@pytest.mark.parametrize("m,B", [(1, 64), (64, 64), (150, 64), (37, 8), (200, 16)])
@pytest.mark.parametrize("average", [True, False])
def test_blocked_inner_loop_equals_stepwise_oracle(m, B, average):
    rng = np.random.default_rng(1000 + m + B)
    N, d = 70, 12
    Z = rng.standard_normal((N, d)) / np.sqrt(d)
    yz = rng.standard_normal(N)
    gamma = rng.uniform(0.5, 2.0, N)
    idx = rng.integers(0, N, m)
    inv_nq = rng.uniform(0.5, 1.5, m)
    w_bar = rng.standard_normal(d) * 0.1
    mu = rng.standard_normal(d) * 1e-2
    eta = 0.3 / np.mean(gamma * np.sum(Z * Z, axis=1))
    ref = svrg.epoch_scaled(Z, yz, gamma, w_bar, idx, inv_nq, eta, average, v_bar=mu)
    got = _blocked_epoch(Z, gamma, w_bar, idx, inv_nq, eta, mu, B, average)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-13)


def test_blocked_form_with_a_dropped_term_fails():
    """The check has teeth: leaving out the mu contribution j . h of the earlier steps in a block
    (an easy slip in the derivation) moves the result well outside the tolerance."""
    rng = np.random.default_rng(7)
    N, d, m, B = 40, 8, 64, 64
    Z = rng.standard_normal((N, d)) / np.sqrt(d)
    gamma = np.ones(N)
    idx = rng.integers(0, N, m)
    inv_nq = np.ones(m)
    w_bar = rng.standard_normal(d) * 0.1
    mu = rng.standard_normal(d) * 0.5
    eta = 0.2
    ref = svrg.epoch_scaled(Z, np.zeros(N), gamma, w_bar, idx, inv_nq, eta, True, v_bar=mu)
    # same blocked form without the -eta (j . h) right-hand side
    delta = np.zeros(d)
    run = np.zeros(d)
    Zb = Z[idx]
    G = Zb @ Zb.T
    R = np.stack([_forward_subst(G, gamma[idx] * inv_nq, eta, np.eye(m)[c]) for c in range(m)], axis=1)
    a = R @ (Zb @ delta)
    jv = np.arange(m, dtype=np.float64)
    run += m * delta - eta * (m * (m + 1) / 2 * mu + ((m - jv) * a) @ Zb)
    wrong = w_bar + run / m
    assert np.linalg.norm(wrong - ref) > 1e-6 * np.linalg.norm(ref)
