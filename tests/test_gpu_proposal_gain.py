"""What the trained proposal network gains over the method without it: on held-out problems (drawn
outside the training records), Alg. 3 with the network's (k, eta, m) reaches relative
suboptimality 1e-6 sooner than with the theory-set parameters of Sec. 3 / Thm 1 and than with the
fixed practice setting (k = 64, eta = 1/beta^, m = 2n), and it is not slower than the constant
setting at the training set's mean parameters (the best single setting the records give without
looking at the problem)."""

import math
import os

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import ridge
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(rs.__file__), "proposal_weights.npz")
PROBLEMS = [(32768, 512, 2.0, 1e-5, 9001), (24576, 256, 1.6, 1e-4, 9002)]


def _weights():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained proposal weights in the package")
    W = np.load(WEIGHTS)
    return torch.from_numpy(W["theta"]).float().cuda(), rs.mlp_norm(W["in_mean"], W["in_std"], W["out_mean"],
                                                                    W["out_std"])


def _time_to_target(solve, m, Xd, yd, lam, ws, cap_steps):
    """(ms, epochs) of solve(epochs, snapshots) to rel. suboptimality 1e-6, or (inf, epochs run)."""
    if m > cap_steps:
        return float("inf"), 0
    epochs = int(max(1, min(60, cap_steps // max(1, m))))
    _, info = solve(epochs, True)
    rel = [ridge.rel_suboptimality(Xd, yd, lam, s.double().cpu().numpy(), ws) for s in info["snapshots"]]
    hit = [i for i, r in enumerate(rel) if r <= 1e-6]
    if not hit:
        return float("inf"), epochs
    e = hit[0] + 1
    solve(e, False)                                            # warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    solve(e, False)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b), e


def _problem(n, d, alpha, lam, seed):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -alpha, 0.05, seed)
    Xf, yf = X.float(), y.float()
    Xd, yd = Xf.double().numpy(), yf.double().numpy()
    return cuda_rows(Xf), yf.cuda(), Xd, yd, ridge.closed_form(Xd, yd, lam)


def _proposed(ctx, X, y, lam, theta, norm):
    def solve(epochs, snapshots):
        return rs.rs_solve_proposed(ctx, X, y, lam, epochs, 5, 6, theta=theta, norm=norm, snapshots=snapshots)
    return solve, rs.rs_solve_proposed(ctx, X, y, lam, 0, 5, 6, theta=theta, norm=norm)[1]


def _fixed(ctx, X, y, lam, k, eta_mult, m):
    def solve(epochs, snapshots):
        return rs.rs_solve(ctx, X, y, k, lam, epochs, 5, 6, m=m, eta_mult=eta_mult, snapshots=snapshots)
    return solve


@pytest.mark.parametrize("n,d,alpha,lam,seed", PROBLEMS)
def test_network_beats_theory_setting(rsctx, n, d, alpha, lam, seed):
    theta, norm = _weights()
    X, y, Xd, yd, ws = _problem(n, d, alpha, lam, seed)
    net, i_net = _proposed(rsctx, X, y, lam, theta, norm)
    th, i_th = _proposed(rsctx, X, y, lam, None, None)
    assert not i_net["fallback"] and i_th["fallback"]
    t_net, e_net = _time_to_target(net, i_net["m"], Xd, yd, lam, ws, 64 * n)
    t_th, _ = _time_to_target(th, i_th["m"], Xd, yd, lam, ws, 64 * n)
    assert np.isfinite(t_net), (i_net, e_net)
    assert t_net < t_th, (t_net, t_th, i_net, i_th)


@pytest.mark.parametrize("n,d,alpha,lam,seed", PROBLEMS)
def test_network_beats_practice_setting(rsctx, n, d, alpha, lam, seed):
    theta, norm = _weights()
    X, y, Xd, yd, ws = _problem(n, d, alpha, lam, seed)
    net, i_net = _proposed(rsctx, X, y, lam, theta, norm)
    t_net, _ = _time_to_target(net, i_net["m"], Xd, yd, lam, ws, 64 * n)
    t_pr, e_pr = _time_to_target(_fixed(rsctx, X, y, lam, 64, 1.0, 2 * n), 2 * n, Xd, yd, lam, ws, 64 * n)
    assert np.isfinite(t_pr), e_pr
    assert t_net < t_pr, (t_net, t_pr, i_net)


def test_network_not_slower_than_constant_setting(rsctx):
    """Against the constant setting the network's edge is small (median 1.12x over the 128 held-out
    problems of the committed evaluation), so it is checked where that evaluation measured it: on
    three further problems of the evaluation recipe (n = 131072, d = 2048, power-law spectra),
    summed, the network is not slower than the constant setting by more than 10%."""
    from paper_1602_02350_gb300 import proposal as pr
    theta, norm = _weights()
    om = np.asarray(norm.out_mean, np.float64)
    rng = np.random.default_rng(4242)
    tn, tc = [], []
    for _ in range(3):
        spec = pr.draw_problem(rng, n_range=(131072, 131072), d_choices=(2048,))
        X, y = pr.make_data(spec)
        n, lam = spec["n"], spec["lam"]
        ref = pr.Reference(X, y, lam)

        def timed(solve, m):
            if m > 64 * n:
                return float("inf")
            epochs = int(max(1, min(60, 64 * n // max(1, m))))
            rel = ref.rel(solve(epochs, True)[1]["snapshots"])
            hit = [i for i, r in enumerate(rel) if r <= 1e-6]
            if not hit:
                return float("inf")
            solve(hit[0] + 1, False)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            solve(hit[0] + 1, False)
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        net, i_net = _proposed(rsctx, X, y, lam, theta, norm)
        tn.append(timed(net, i_net["m"]))
        k, em, m = int(min(64, max(1, round(2.0 ** om[0])))), float(math.exp(om[1])), int(round(n * 2.0 ** om[2]))
        tc.append(timed(_fixed(rsctx, X, y, lam, k, em, m), m))
        del X, y, ref
        torch.cuda.empty_cache()
    assert all(np.isfinite(tn)), tn
    assert sum(tn) <= 1.1 * sum(tc), (tn, tc)
