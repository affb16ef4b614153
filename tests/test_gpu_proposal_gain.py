"""What the trained proposal network gains over the method without it: on held-out problems (drawn
outside the training records), Alg. 3 with the network's (k, eta, m) reaches relative
suboptimality 1e-6 sooner than with the theory-set parameters of Sec. 3 / Thm 1."""

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


def _weights():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained proposal weights in the package")
    W = np.load(WEIGHTS)
    return torch.from_numpy(W["theta"]).float().cuda(), rs.mlp_norm(W["in_mean"], W["in_std"], W["out_mean"],
                                                                    W["out_std"])


def _time_to_target(ctx, X, y, lam, Xd, yd, ws, theta, norm, cap_steps):
    """(ms, epochs) of rs_solve_proposed to rel. suboptimality 1e-6, or (inf, epochs run)."""
    n = X.shape[0]
    _, info = rs.rs_solve_proposed(ctx, X, y, lam, 1, 5, 6, theta=theta, norm=norm)
    epochs = int(max(1, min(60, cap_steps // max(1, info["m"]))))
    if info["m"] > cap_steps:
        return float("inf"), 0, info
    _, info = rs.rs_solve_proposed(ctx, X, y, lam, epochs, 5, 6, theta=theta, norm=norm, snapshots=True)
    rel = [ridge.rel_suboptimality(Xd, yd, lam, s.double().cpu().numpy(), ws) for s in info["snapshots"]]
    hit = [i for i, r in enumerate(rel) if r <= 1e-6]
    if not hit:
        return float("inf"), epochs, info
    e = hit[0] + 1
    rs.rs_solve_proposed(ctx, X, y, lam, e, 5, 6, theta=theta, norm=norm)       # warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    rs.rs_solve_proposed(ctx, X, y, lam, e, 5, 6, theta=theta, norm=norm)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b), e, info


@pytest.mark.parametrize("n,d,alpha,lam,seed", [(32768, 512, 2.0, 1e-5, 9001), (24576, 256, 1.6, 1e-4, 9002)])
def test_network_beats_theory_setting(rsctx, n, d, alpha, lam, seed):
    theta, norm = _weights()
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -alpha, 0.05, seed)
    Xf, yf = X.float(), y.float()
    Xd, yd = Xf.double().numpy(), yf.double().numpy()
    ws = ridge.closed_form(Xd, yd, lam)
    Xc, yc = cuda_rows(Xf), yf.cuda()
    t_net, e_net, i_net = _time_to_target(rsctx, Xc, yc, lam, Xd, yd, ws, theta, norm, 64 * n)
    t_th, e_th, i_th = _time_to_target(rsctx, Xc, yc, lam, Xd, yd, ws, None, None, 64 * n)
    assert not i_net["fallback"] and i_th["fallback"]
    assert np.isfinite(t_net), (i_net, e_net)
    assert t_net < t_th, (t_net, t_th, i_net["k"], i_net["eta_mult"], i_net["m"], i_th["k"], i_th["m"])
