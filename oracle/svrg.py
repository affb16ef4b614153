"""SVRG with importance sampling (Alg. 1, the Xiao-Zhang variant of Sec. 4.2) on the
n+d preconditioned components of Sec. 5.1, float64 (oracle; test infrastructure).

F(w) = (1/N) sum_i f_i(w) with f_i(w) = gamma_i 1/2 (z_i^T w - y_i)^2 (see
``precond.components``).  The variance-reduced direction is read as
    v_t = (grad f_i(w_{t-1}) - grad f_i(w_bar)) / (N q_i) + v_bar,
the unbiased form for an average of N functions (Alg. 1 prints the division by
q_i without the 1/N).
"""

import numpy as np

from . import streams


def grad_component(Z, yz, gamma, i, w):
    """grad f_i(w) = gamma_i (z_i^T w - y_i) z_i."""
    z = Z[i]
    return gamma[i] * (z @ w - yz[i]) * z


def full_gradient(Z, yz, gamma, w):
    """grad F(w) = (1/N) sum_i grad f_i(w) (Alg. 1, v_bar).  For the components of
    Sec. 5.1 this equals X~^T (X~ w - y) / n + lam M^T M w."""
    N = Z.shape[0]
    g = np.zeros(Z.shape[1])
    for i in range(N):
        g += grad_component(Z, yz, gamma, i, w)
    return g / N


def full_gradient_fast(Z, yz, gamma, w):
    """Same value as ``full_gradient`` as one matrix expression (for large N)."""
    r = gamma * (Z @ w - yz)
    return Z.T @ r / Z.shape[0]


def full_gradient_chunked(chunks, N, w):
    """``full_gradient_fast`` over row blocks (Z_b, yz_b, gamma_b) given in any split, for N rows
    in total: (1/N) sum_b Z_b^T (gamma_b (Z_b w - yz_b)), each block converted to float64."""
    g = None
    w = np.asarray(w, np.float64)
    for Zb, yb, gb in chunks:
        Zb = np.asarray(Zb, np.float64)
        r = np.asarray(gb, np.float64) * (Zb @ w - np.asarray(yb, np.float64))
        g = Zb.T @ r if g is None else g + Zb.T @ r
    return g / N


def epoch(Z, yz, gamma, w_bar, idx, q, eta, average=True, v_bar=None):
    """One outer iteration s of Alg. 1 for a given index stream i_1..i_m.

    w_0 = w_bar; w_t = w_{t-1} - eta v_t; returns (1/m) sum_{t=1..m} w_t
    (or w_m when ``average`` is False, the last-iterate option).
    """
    N = Z.shape[0]
    inv_nq = 1.0 / (N * np.asarray(q, np.float64)[np.asarray(idx)])
    return epoch_scaled(Z, yz, gamma, w_bar, idx, inv_nq, eta, average, v_bar)


def epoch_scaled(Z, yz, gamma, w_bar, idx, inv_nq, eta, average=True, v_bar=None):
    """Alg. 1's inner loop with the factor 1/(N q_{i_t}) of each step given explicitly
    (``inv_nq[t]``), so that any index stream and weights can be replayed."""
    if v_bar is None:
        v_bar = full_gradient_fast(Z, yz, gamma, w_bar)
    w = np.array(w_bar, np.float64)
    acc = np.zeros_like(w)
    for t, i in enumerate(idx):
        v = (grad_component(Z, yz, gamma, i, w) - grad_component(Z, yz, gamma, i, w_bar)) * inv_nq[t] + v_bar
        w = w - eta * v
        acc += w
    return acc / len(idx) if average else w


def sampling_table(beta):
    """(W, cum, q): integer weights, their prefix sums and q_i = W_i / sum W."""
    W = streams.quantize_weights(beta)
    cum = streams.cumulative(W)
    q = W.astype(np.float64) / float(cum[-1])
    return W, cum, q


def solve(Z, yz, gamma, beta, eta, m, epochs, seed, w0=None, epoch0=0,
          uniform=False, average=True, callback=None):
    """Alg. 1 for ``epochs`` outer iterations, starting at ``w0`` (zero if None).

    Epoch s (counted from ``epoch0``, which lets a run resume at an epoch
    boundary) draws its indices from the Philox stream of (seed, s).
    Returns the list of snapshots w_bar_1..w_bar_S.
    """
    N, d = Z.shape
    W, cum, q = sampling_table(beta)
    if uniform:
        q = np.full(N, 1.0 / N)
    w_bar = np.zeros(d) if w0 is None else np.array(w0, np.float64)
    snaps = []
    for s in range(epoch0, epoch0 + epochs):
        if uniform:
            idx = streams.sample_indices_uniform(N, seed, s, m)
        else:
            idx = streams.sample_indices(cum, seed, s, m)
        w_bar = epoch(Z, yz, gamma, w_bar, idx, q, eta, average)
        snaps.append(w_bar.copy())
        if callback is not None:
            callback(s, w_bar)
    return snaps
