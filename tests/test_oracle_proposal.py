"""Pins for oracle.proposal: backpropagation against central differences and against torch
autograd, the forward pass and Adam against torch's own modules, and the theory defaults
against the preconditioner oracle (Thm 4 trace identity) and a two-level spectrum whose
optimal rank is known in closed form."""

import numpy as np
import pytest
import torch

from oracle import precond, proposal, ridge
from paper_1602_02350_gb300 import synth


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, proposal.IN)), rng.standard_normal((B, proposal.OUT))


def _torch_net(theta):
    W1, b1, W2, b2, W3, b3 = [torch.tensor(a, dtype=torch.float64) for a in proposal.unpack(theta)]
    net = torch.nn.Sequential(torch.nn.Linear(67, 128), torch.nn.ReLU(), torch.nn.Linear(128, 128), torch.nn.ReLU(),
                              torch.nn.Linear(128, 3)).double()
    with torch.no_grad():
        for lin, (W, b) in zip([net[0], net[2], net[4]], [(W1, b1), (W2, b2), (W3, b3)]):
            lin.weight.copy_(W)
            lin.bias.copy_(b)
    return net


def test_layout_and_init():
    theta = synth.mlp_init(1)
    assert theta.shape == (proposal.NPARAM,) == (25603,)
    W1, b1, W2, b2, W3, b3 = proposal.unpack(theta)
    assert W1.shape == (128, 67) and W3.shape == (3, 128) and not b2.any()


def test_forward_matches_torch_modules():
    theta = synth.mlp_init(2)
    X, _ = _batch(17, 3)
    out, _ = proposal.forward(theta, X)
    ref = _torch_net(theta)(torch.tensor(X)).detach().numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_gradient_matches_autograd():
    theta = synth.mlp_init(4)
    theta[proposal.NPARAM - 3:] = [0.3, -0.2, 0.1]
    X, T = _batch(9, 5)
    L, g = proposal.gradient(theta, X, T)
    net = _torch_net(theta)
    out = net(torch.tensor(X))
    Lt = ((out - torch.tensor(T)) ** 2).sum() / X.shape[0]
    Lt.backward()
    gt = np.concatenate([p.grad.numpy().ravel() for p in net.parameters()])
    assert L == pytest.approx(Lt.item(), rel=1e-13)
    np.testing.assert_allclose(g, gt, rtol=1e-11, atol=1e-13)


def test_gradient_matches_central_differences():
    theta = synth.mlp_init(6)
    X, T = _batch(5, 7)
    _, g = proposal.gradient(theta, X, T)
    rng = np.random.default_rng(8)
    h = 1e-6
    for p in list(rng.choice(proposal.NPARAM, 40, replace=False)) + [proposal.NPARAM - 1, 128 * 67]:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (proposal.loss(proposal.forward(tp, X)[0], T) - proposal.loss(proposal.forward(tm, X)[0], T)) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=1e-5, abs=1e-8), p


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(9)
    theta = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.8, 0.99), eps=1e-6)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        theta, m, v = proposal.adam_step(theta, m, v, g, t, lr=3e-3, beta1=0.8, beta2=0.99, eps=1e-6)
        p.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, _, _ = proposal.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(th, [-0.01, 0.01, -0.01, 0.0], rtol=1e-8)


def test_kappa_model_is_the_smoothness_of_exactly_preconditioned_components():
    """With V the exact leading eigenvectors, the mean smoothness of the M-scaled components
    (computed by the preconditioner oracle row by row) equals lam (kappa~(k) + d)."""
    n, d, lam = 400, 24, 1e-3
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -1.7, 0.1, 11)
    X = X.numpy()
    C = ridge.correlation(X)
    ev, U = np.linalg.eigh(C)
    ev, U = ev[::-1], U[:, ::-1]
    trc = np.trace(C)
    assert trc == pytest.approx((X * X).sum() / n, rel=1e-12)
    for k in (1, 3, 8, 24):
        M = precond.m_matrix(U[:, :k], ev[:k], lam)
        Z, _, g = precond.components(*precond.transform(X, M), y.numpy(), lam)
        bh = precond.beta_hat(precond.smoothness(Z, g))
        assert bh == pytest.approx(proposal.beta_hat_model(ev, trc, lam, k, d), rel=1e-10)
        assert bh / lam == pytest.approx(proposal.kappa_tilde(ev, trc, lam, k) + d, rel=1e-10)


@pytest.mark.parametrize("n,expect_rank_plus_one", [(50, True), (5000, False)])
def test_theory_rank_on_two_level_spectrum(n, expect_rank_plus_one):
    """r eigenvalues a, the rest b < a: kappa~ is flat in k <= r and drops to d b / lam at
    k = r + 1, so the model picks r + 1 exactly when n < (a - b) / lam, else 1."""
    d, r, a, b, lam = 100, 5, 1.0, 1e-3, 1e-3   # (a - b) / lam = 999
    s = np.array([a] * r + [b] * (d - r))
    k = proposal.theory_rank(s, s.sum(), lam, n, d)
    assert k == (r + 1 if expect_rank_plus_one else 1)
    k2, em, m = proposal.theory_defaults(s, s.sum(), lam, n, d)
    assert (k2, em) == (k, 0.1)
    assert m == int(np.ceil(proposal.kappa_tilde(s, s.sum(), lam, k) + d))


def test_features():
    s2 = 4.0 * np.geomspace(1.0, 1e-8, 70)
    f = proposal.features(s2, 1e-5, 1000, 64)
    assert f.shape == (67,)
    np.testing.assert_allclose(f[:64], 0.5 * np.log(s2[:64] / 4.0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(f[64:], np.log([1e-5 / 4.0, 1000, 64]), rtol=1e-14)


def test_features_are_scale_invariant():
    # X -> c X scales the sketched spectrum and the equivalent lam by c^2: the input does not change
    s2 = np.geomspace(3.0, 3e-6, 64)
    np.testing.assert_allclose(proposal.features(s2, 1e-4, 5000, 256), proposal.features(49.0 * s2, 49e-4, 5000, 256),
                               rtol=1e-12, atol=1e-12)


def test_network_input_clips_to_the_training_spread():
    x = np.array([0.0, 5.0, -7.0, 1.0])
    z = proposal.network_input(x, np.zeros(4), np.array([1.0, 1.0, 2.0, 0.5]))
    np.testing.assert_array_equal(z, [0.0, proposal.INPUT_CLIP, -proposal.INPUT_CLIP, 2.0])
