"""GPU parity of the proposal network (forward, backpropagation, Adam) against the oracle, and of
rs_propose against the theory-set parameters of Sec. 3 / Thm 1."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import proposal
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


def _f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).float()


def _batch(B, seed, margin=1e-4, theta=None):
    """Inputs and targets; with theta, samples whose pre-activations come within `margin` of the
    ReLU kink are dropped (FP32 and FP64 could take different sides there)."""
    rng = np.random.default_rng(seed)
    X = _f32(rng.standard_normal((B, 67))).double().numpy()
    T = _f32(rng.standard_normal((B, 3))).double().numpy()
    if theta is not None:
        _, (_, a1, _, a2, _) = proposal.forward(theta, X)
        keep = (np.abs(a1).min(1) > margin) & (np.abs(a2).min(1) > margin)
        X, T = X[keep], T[keep]
    return X, T


def _theta(seed):
    return _f32(synth.mlp_init(seed)).double().numpy()


@pytest.mark.parametrize("B", [1, 31, 32, 33, 1000])
def test_forward_matches_oracle(rsctx, B):
    theta = _theta(B)
    X, _ = _batch(B, B + 1)
    out = rs.rs_mlp_forward(rsctx, _f32(theta).cuda(), _f32(X).cuda()).cpu().double().numpy()
    ref, _ = proposal.forward(theta, X)
    np.testing.assert_allclose(out, ref, rtol=0, atol=2e-5 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("B", [1, 7, 32, 100, 2048])
def test_train_step_gradient_and_adam_match_oracle(rsctx, B):
    theta = _theta(3 * B)
    X, T = _batch(B, B + 5, theta=theta)
    th = _f32(theta).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    g, loss = rs.rs_mlp_train_step(rsctx, th, m, v, _f32(X).cuda(), _f32(T).cuda(), 1, lr=1e-3, want_grad=True)
    L_ref, g_ref = proposal.gradient(theta, X, T)
    assert loss.item() == pytest.approx(L_ref, rel=1e-5)
    g = g.cpu().double().numpy()
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-5 * np.abs(g_ref).max())
    # Adam from the GPU gradient (the update divides by |g|, so it is compared for the same g)
    # the kernel holds the hyper-parameters in float: give the oracle the same values
    f = lambda v: float(np.float32(v))  # noqa: E731
    th_ref, m_ref, v_ref = proposal.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), g, 1, lr=f(1e-3),
                                              beta1=f(0.9), beta2=f(0.999), eps=f(1e-8))
    # theta is stored in float: the updated value is the FP64 one rounded once (half an ulp)
    np.testing.assert_allclose(th.cpu().double().numpy(), th_ref, rtol=2.0 ** -23, atol=1e-9)
    np.testing.assert_allclose(m.cpu().double().numpy(), m_ref, rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(v.cpu().double().numpy(), v_ref, rtol=1e-5, atol=1e-16)


def test_several_steps_track_the_oracle(rsctx):
    theta = _theta(42)
    th = _f32(theta).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    tr, mr, vr = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 6):
        X, T = _batch(256, 100 + t, theta=tr)
        rs.rs_mlp_train_step(rsctx, th, m, v, _f32(X).cuda(), _f32(T).cuda(), t, lr=1e-3)
        _, g = proposal.gradient(tr, X, T)
        tr, mr, vr = proposal.adam_step(tr, mr, vr, g, t, lr=1e-3)
    # each Adam step moves a parameter by at most about lr: FP32 drift stays far below that
    np.testing.assert_allclose(th.cpu().double().numpy(), tr, rtol=0, atol=2e-4)


def test_training_fits_a_smooth_target(rsctx):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((67, 3)) / np.sqrt(67)
    th = _f32(synth.mlp_init(8)).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    losses = []
    for t in range(1, 401):
        X = rng.standard_normal((512, 67))
        T = np.tanh(X @ A)
        _, loss = rs.rs_mlp_train_step(rsctx, th, m, v, _f32(X).cuda(), _f32(T).cuda(), t, lr=2e-3)
        losses.append(loss.item())
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5]), (losses[:5], losses[-20:])


def _spectrum(d, alpha, seed):
    rng = np.random.default_rng(seed)
    s = np.arange(1, d + 1, dtype=np.float64) ** -alpha * np.exp(0.1 * rng.standard_normal(d))
    return np.sort(s)[::-1]


@pytest.mark.parametrize("n,d,alpha,lam", [(65536, 1024, 2.0, 1e-5), (16384, 256, 1.2, 1e-3), (262144, 4096, 2.5, 1e-7),
                                          (100, 64, 1.0, 1e-2)])
def test_propose_fallback_is_the_theory_setting(rsctx, n, d, alpha, lam):
    s = _spectrum(d, alpha, n)
    k, em, m, fb = rs.rs_propose(rsctx, s[:64], lam, n, d, s.sum())
    assert fb
    assert (k, em, m) == proposal.theory_defaults(s[:64], s.sum(), lam, n, d)


def _norm():
    rng = np.random.default_rng(3)
    return (rng.uniform(-3, 0, 67), rng.uniform(0.5, 2, 67), np.array([4.0, 0.0, -1.0]), np.array([1.0, 0.5, 1.0]))


def _proposal_theta(bias):
    theta = synth.mlp_init(11) * 0.05
    theta[proposal.NPARAM - 3:] = bias
    return _f32(theta).double().numpy()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_propose_runs_the_network(rsctx, seed):
    n, d, lam = 131072, 2048, 1e-6
    s = _spectrum(d, 1.5, seed)
    theta = _proposal_theta([0.3, 0.2, -0.5])
    im, isd, om, osd = _norm()
    nm = rs.mlp_norm(im, isd, om, osd)
    k, em, m, fb = rs.rs_propose(rsctx, s[:64], lam, n, d, s.sum(), theta=_f32(theta).cuda(), norm=nm)
    assert not fb
    x = proposal.network_input(proposal.features(s[:64], lam, n, d), _f32(im).double().numpy(),
                               _f32(isd).double().numpy())
    o, _ = proposal.forward(theta, x[None, :])
    o = o[0] * _f32(osd).double().numpy() + _f32(om).double().numpy()
    assert k == int(np.clip(np.round(2.0 ** o[0]), 1, 64))
    assert em == pytest.approx(np.exp(o[1]), rel=1e-4)
    assert m == pytest.approx(n * 2.0 ** o[2], rel=1e-4)


def test_propose_falls_back_outside_the_training_box(rsctx):
    n, d, lam = 131072, 2048, 1e-6
    s = _spectrum(d, 1.5, 5)
    im, isd, om, osd = _norm()
    nm = rs.mlp_norm(im, isd, om, osd)
    theta = _proposal_theta([0.0, 12.0, 0.0])     # eta_mult = e^6: outside [0.01, 8]
    k, em, m, fb = rs.rs_propose(rsctx, s[:64], lam, n, d, s.sum(), theta=_f32(theta).cuda(), norm=nm)
    assert fb and (k, em, m) == proposal.theory_defaults(s[:64], s.sum(), lam, n, d)


def test_propose_rejects_bad_spectra(rsctx):
    s = np.linspace(1.0, 2.0, 64)                  # ascending
    with pytest.raises(rs.RsError):
        rs.rs_propose(rsctx, s, 1e-3, 100, 64, 1.0)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_trace_c_matches_oracle(rsctx, dtype):
    from oracle import ridge
    from tests.gpu_helpers import cuda_rows
    X = torch.from_numpy(synth.random_matrix(3001, 70, 4)).to(dtype)
    tr = rs.rs_trace_c(rsctx, cuda_rows(X))
    # lanes sum their part of a row in float (float data) before the double accumulation
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    assert tr == pytest.approx(np.trace(ridge.correlation(X.double().numpy())), rel=tol)


@pytest.mark.parametrize("z_dtype", [None, torch.bfloat16])
def test_solve_proposed_equals_its_steps(rsctx, z_dtype):
    """rs_solve_proposed = rank-64 sketch, tr(C), rs_propose, leading-k components, SVRG, bit for bit;
    host buffers give the same result as device buffers."""
    from tests.gpu_helpers import cuda_rows
    n, d, lam = 6000, 128, 1e-4
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.6, 0.1, 31)
    Xc, yc = cuda_rows(X.float()), y.float().cuda()
    im, isd, om, osd = _norm()
    nm = rs.mlp_norm(im, isd, om, osd)
    theta = _f32(_proposal_theta([0.3, 0.2, -0.5])).cuda()
    w, info = rs.rs_solve_proposed(rsctx, Xc, yc, lam, 3, 11, 12, theta=theta, norm=nm, z_dtype=z_dtype)
    V, s2 = rs.rs_sketch(rsctx, Xc, 64, 11)
    k, em, m, fb = rs.rs_propose(rsctx, s2.cpu().numpy(), lam, n, d, rs.rs_trace_c(rsctx, Xc), theta=theta, norm=nm)
    assert (k, m, fb) == (info["k"], info["m"], info["fallback"]) and em == info["eta_mult"]
    Vk, s2k = V[:, :k].contiguous(), s2[:k].contiguous()
    Z, beta, _ = rs.rs_precondition(rsctx, Xc, Vk, s2k, lam, z_dtype=z_dtype)
    w2, _ = rs.rs_svrg_solve(rsctx, Z, yc, Vk, s2k, lam, 3, 12, beta=beta, m=m, eta_mult=em,
                             X=Xc if z_dtype is not None else None, refine=z_dtype is not None)
    assert torch.equal(w, w2)
    Xh = Xc.cpu().pin_memory()
    wh, _ = rs.rs_solve_proposed(rsctx, Xh, yc.cpu().pin_memory(), lam, 3, 11, 12, theta=theta, norm=nm,
                                 z_dtype=z_dtype, w_out=torch.empty(d).pin_memory())
    assert torch.equal(wh, w.cpu())


@pytest.mark.parametrize("z_dtype", [None, torch.bfloat16])
def test_solve_proposed_with_fixed_rank_equals_its_steps(rsctx, z_dtype):
    """With a caller-fixed rank k > 64 the features are the first 64 Ritz values of the rank-k sketch,
    the preconditioner keeps all k pairs and only (eta, m) come from the network, bit for bit."""
    from tests.gpu_helpers import cuda_rows
    n, d, lam, kf = 6000, 192, 1e-4, 96
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.4, 0.1, 33)
    Xc, yc = cuda_rows(X.float()), y.float().cuda()
    im, isd, om, osd = _norm()
    nm = rs.mlp_norm(im, isd, om, osd)
    theta = _f32(_proposal_theta([0.3, 0.2, -0.5])).cuda()
    w, info = rs.rs_solve_proposed(rsctx, Xc, yc, lam, 3, 11, 12, theta=theta, norm=nm, z_dtype=z_dtype, k_fixed=kf)
    assert info["k"] == kf
    V, s2 = rs.rs_sketch(rsctx, Xc, kf, 11)
    trc = rs.rs_trace_c(rsctx, Xc)
    kn, em, m, fb = rs.rs_propose(rsctx, s2[:64].cpu().numpy(), lam, n, d, trc, theta=theta, norm=nm)
    assert not fb
    # the network's epoch length carried to the fixed rank by kappa~(k_fixed) / kappa~(k_net) (Thm 1)
    s2n = s2.cpu().numpy()
    m = max(1, int(np.floor(m * proposal.kappa_tilde(s2n, trc, lam, kf) / proposal.kappa_tilde(s2n, trc, lam, kn) + 0.5)))
    assert (m, fb) == (info["m"], info["fallback"]) and em == info["eta_mult"]
    Z, beta, _ = rs.rs_precondition(rsctx, Xc, V, s2, lam, z_dtype=z_dtype)
    w2, _ = rs.rs_svrg_solve(rsctx, Z, yc, V, s2, lam, 3, 12, beta=beta, m=m, eta_mult=em,
                             X=Xc if z_dtype is not None else None, refine=z_dtype is not None)
    assert torch.equal(w, w2)


def test_solve_proposed_without_weights_uses_the_theory_setting(rsctx):
    from tests.gpu_helpers import cuda_rows
    n, d, lam = 4000, 96, 1e-3
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.3, 0.1, 32)
    Xc = cuda_rows(X.float())
    _, info = rs.rs_solve_proposed(rsctx, Xc, y.float().cuda(), lam, 1, 3, 4)
    V, s2 = rs.rs_sketch(rsctx, Xc, 64, 3)
    th = proposal.theory_defaults(s2.cpu().numpy(), rs.rs_trace_c(rsctx, Xc), lam, n, d)
    assert info["fallback"] and (info["k"], info["eta_mult"], info["m"]) == th
