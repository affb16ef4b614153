"""Parameter proposal: the theory-set defaults of Sec. 3 / Thm 1 and the proposal network
(a multilayer perceptron 67 -> 128 -> 128 -> 3 with ReLU) that replaces them, float64
(oracle; test infrastructure).

Theory defaults.  The SVRG theorem quoted in Sec. 3 (Xiao and Zhang) runs Alg. 1 with
eta = 0.1 / beta^ and m = ceil(kappa^_F), kappa^_F = beta^ / alpha (Eq. (5) notation).
For the M-preconditioned components beta^ = tr(M (C + lam I) M) (Thm 4 trace identity,
pinned in test_oracle_precond) and alpha >= lam, so the defaults use kappa^_F = beta^ / lam.
With V the exact leading eigenvectors, tr(M (C + lam I) M) = k sigma_k^2 + sum_{i>k} sigma_i^2
+ d lam, i.e. kappa^_F = kappa~(k) + d with kappa~ the average condition number of Thm 1.
The rank k minimises the runtime model of Thm 1: preconditioning n d k plus
(kappa~(k) + n + d) d per factor of accuracy, over k = 1..min(64, d).

Network.  Not in the paper: it maps the log of the 64 leading sketched singular values
(square roots of sigma~_i^2), log lam, log n and log d to (log2 k, ln eta_mult, log2(m / n)),
where the step size is eta = eta_mult / beta^.  Inputs and outputs are normalised by fixed
affine maps stored with the weights.  Parameters are one flat vector:
W1 (128 x 67), b1 (128), W2 (128 x 128), b2 (128), W3 (3 x 128), b3 (3), row-major.
Loss: mean over the batch of the squared error summed over the 3 outputs.  Optimiser:
Adam (Kingma and Ba, ICLR 2015) with bias correction.
"""

import numpy as np

IN, HID, OUT = 67, 128, 3
SHAPES = [(HID, IN), (HID,), (HID, HID), (HID,), (OUT, HID), (OUT,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)


# ------------------------------------------------------------------ theory defaults

def kappa_tilde(sigma2, trace_c, lam, k):
    """Thm 1: kappa~(k) = (k sigma_k^2 + sum_{i>k} sigma_i^2) / lam, the tail sum written as
    tr(C) - sum_{i<=k} sigma_i^2 (tr(C) = ||X||_F^2 / n is exact from one pass)."""
    s = np.asarray(sigma2, np.float64)
    return (k * s[k - 1] + (trace_c - s[:k].sum())) / lam


def beta_hat_model(sigma2, trace_c, lam, k, d):
    """tr(M (C + lam I) M) when V holds exact eigenvectors: k (sigma_k^2 + lam) + the tail
    of the spectrum + (d - k) lam = lam (kappa~(k) + d)."""
    return lam * (kappa_tilde(sigma2, trace_c, lam, k) + d)


def theory_rank(sigma2, trace_c, lam, n, d, kmax=64):
    """argmin_k n d k + (kappa~(k) + n + d) d over k = 1..min(kmax, len(sigma2), d)
    (first minimiser on ties)."""
    K = min(kmax, len(sigma2), d)
    cost = [n * d * k + (kappa_tilde(sigma2, trace_c, lam, k) + n + d) * d for k in range(1, K + 1)]
    return int(np.argmin(cost)) + 1


def theory_defaults(sigma2, trace_c, lam, n, d, kmax=64):
    """(k, eta_mult, m) of the theory setting: eta = 0.1 / beta^, m = ceil(beta^ / lam), with
    beta^ / lam = kappa~(k) + d written without the round trip through beta^."""
    k = theory_rank(sigma2, trace_c, lam, n, d, kmax)
    return k, 0.1, int(np.ceil(kappa_tilde(sigma2, trace_c, lam, k) + d))


# ------------------------------------------------------------------ network

def unpack(theta):
    """Views of the flat parameter vector as (W1, b1, W2, b2, W3, b3)."""
    theta = np.asarray(theta)
    out, o = [], 0
    for s in SHAPES:
        c = int(np.prod(s))
        out.append(theta[o:o + c].reshape(s))
        o += c
    return out


def forward(theta, X):
    """Network outputs (B x 3) and the activations the gradient needs."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64))
    X = np.asarray(X, np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ W3.T + b3
    return out, (X, a1, h1, a2, h2)


def loss(out, T):
    """(1/B) sum_s sum_o (out_so - t_so)^2."""
    D = np.asarray(out, np.float64) - np.asarray(T, np.float64)
    return float((D * D).sum() / D.shape[0])


def gradient(theta, X, T):
    """Loss and its gradient with respect to the flat parameter vector (chain rule, layer by
    layer; the ReLU derivative is taken as 0 at 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64))
    out, (X, a1, h1, a2, h2) = forward(theta, X)
    B = X.shape[0]
    g_out = 2.0 * (out - np.asarray(T, np.float64)) / B
    gW3 = g_out.T @ h2
    gb3 = g_out.sum(0)
    g_h2 = g_out @ W3
    g_a2 = g_h2 * (a2 > 0)
    gW2 = g_a2.T @ h1
    gb2 = g_a2.sum(0)
    g_h1 = g_a2 @ W2
    g_a1 = g_h1 * (a1 > 0)
    gW1 = g_a1.T @ X
    gb1 = g_a1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss(out, T), g


def adam_step(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1: returns the new (theta, m, v)."""
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return np.asarray(theta, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def features(sigma2_64, lam, n, d):
    """Network input: log of the 64 leading sketched singular values (sqrt of sigma~_i^2, floored
    at 1e-30) and log lam, both relative to the leading value (log(s_i / s_1), log(lam / s_1^2)), then
    log n, log d.  Scaling X by c scales every sigma~_i^2 and the lam of the equivalent problem by
    c^2 and leaves (k, eta beta^, m) unchanged, so the input is taken invariant to it."""
    s = np.sqrt(np.maximum(np.asarray(sigma2_64, np.float64)[:64], 1e-60))
    ls = np.log(np.maximum(s, 1e-30))
    return np.concatenate([ls - ls[0], [np.log(lam) - 2.0 * ls[0], np.log(n), np.log(d)]])


INPUT_CLIP = 3.0   # normalised inputs are clipped to +-INPUT_CLIP (training spreads) before the network


def network_input(x, in_mean, in_std):
    """(x - in_mean) / in_std, clipped to [-INPUT_CLIP, INPUT_CLIP]: a problem outside the training
    ranges (larger n, a smaller lam) is proposed for as if at their edge instead of extrapolating."""
    return np.clip((np.asarray(x, np.float64) - in_mean) / in_std, -INPUT_CLIP, INPUT_CLIP)
