"""Accelerated SVRG (Catalyst around Alg. 1, rs_catalyst_solve) against the oracle's Catalyst on the
same components, seeds and smoothness constants (trajectory parity in FP64), and convergence to the
ridge solution in FP32 and with BF16 components refined on the stored data."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import catalyst, precond, ridge
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    cfg = synth.CONFIGS["fp64_n4096_d256"]
    X, y, _ = synth.config_problem(cfg)
    Xn, yn = X.numpy(), y.numpy()
    return cfg, X, y, Xn, yn, ridge.closed_form(Xn, yn, cfg.lam)


def test_catalyst_fp64_follows_the_oracle(rsctx, problem):
    cfg, X, y, Xn, yn, ws = problem
    n, d, lam = cfg.n, cfg.d, cfg.lam
    V, s2 = rs.rs_sketch(rsctx, X.cuda(), cfg.k, cfg.seed_sketch)
    Z, beta, _ = rs.rs_precondition(rsctx, X.cuda(), V, s2, lam)
    w, info = rs.rs_catalyst_solve(rsctx, Z, y.cuda(), V, s2, lam, 4, 2, cfg.seed_svrg, beta=beta, m=2048,
                                   eta_mult=1.0, snapshots=True)
    kappa = info["kappa"]
    assert kappa > 0
    M = precond.m_matrix(V.cpu().numpy(), s2.cpu().numpy(), lam)
    Zr, yz, g = precond.components(*precond.transform(Xn, M), yn, lam)
    xs = catalyst.solve(Zr, yz, g, beta.cpu().numpy(), M, n, lam, kappa, 4, 2, 2048, 1.0, cfg.seed_svrg)
    got = info["snapshots"].cpu().numpy()
    for t in range(4):
        err = np.linalg.norm(got[t] - xs[t]) / np.linalg.norm(xs[t])
        assert err <= 1e-9, (t, err)
    np.testing.assert_allclose(w.cpu().numpy(), xs[-1], rtol=1e-9, atol=1e-12)
    # the default kappa is Catalyst's L / N - mu with L the mean smoothness of the original components
    assert kappa == pytest.approx(precond.beta_hat(beta.cpu().numpy()) / (n + d) - lam, rel=1e-12)


def test_catalyst_fp32_converges(rsctx, problem):
    cfg, X, y, Xn, yn, ws = problem
    lam = cfg.lam
    Xf, yf = X.float(), y.float()
    V, s2 = rs.rs_sketch(rsctx, Xf.cuda(), cfg.k, cfg.seed_sketch)
    Z, beta, _ = rs.rs_precondition(rsctx, Xf.cuda(), V, s2, lam)
    _, info = rs.rs_catalyst_solve(rsctx, Z, yf.cuda(), V, s2, lam, 12, 2, 5, beta=beta, m=2 * cfg.n,
                                   eta_mult=1.0, snapshots=True)
    Xd, yd = Xf.double().numpy(), yf.double().numpy()
    wsd = ridge.closed_form(Xd, yd, lam)
    rel = [ridge.rel_suboptimality(Xd, yd, lam, s, wsd) for s in info["snapshots"].double().cpu().numpy()]
    assert rel[-1] <= 1e-7, rel
    assert rel[-1] <= 1e-4 * rel[0], rel


def test_catalyst_bf16_refined_converges(rsctx):
    n, d, k, lam = 8192, 256, 16, 1e-4
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.5, 0.1, 78)
    Xb = cuda_rows(X.to(torch.bfloat16))
    yf = y.float().cuda()
    V, s2 = rs.rs_sketch(rsctx, Xb, k, 3)
    Z, beta, _ = rs.rs_precondition(rsctx, Xb, V, s2, lam)
    _, info = rs.rs_catalyst_solve(rsctx, Z, yf, V, s2, lam, 10, 2, 7, beta=beta, m=2 * n, eta_mult=1.0, X=Xb,
                                   refine=True, snapshots=True)
    Xd = X.to(torch.bfloat16).double().numpy()
    yd = yf.double().cpu().numpy()
    wsd = ridge.closed_form(Xd, yd, lam)
    rel = [ridge.rel_suboptimality(Xd, yd, lam, s, wsd) for s in info["snapshots"].double().cpu().numpy()]
    assert rel[-1] <= 1e-7, rel


def test_catalyst_rejects_bad_arguments(rsctx, problem):
    cfg, X, y, *_ = problem
    V, s2 = rs.rs_sketch(rsctx, X.cuda(), cfg.k, cfg.seed_sketch)
    Z, beta, _ = rs.rs_precondition(rsctx, X.cuda(), V, s2, cfg.lam)
    for outer, epochs in ((0, 1), (2, 0)):
        with pytest.raises(rs.RsError) as e:
            rs.rs_catalyst_solve(rsctx, Z, y.cuda(), V, s2, cfg.lam, outer, epochs, 1, beta=beta, m=100)
        assert e.value.code == 1
