"""End-to-end parity (Alg. 3) on the FP64 workload and the FP32 CountSketch workload at full size,
plus the objective, resume and error paths, all through the C ABI."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import pipeline, precond, ridge, streams
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp64_problem():
    cfg = synth.CONFIGS["fp64_n4096_d256"]
    X, y, _ = synth.config_problem(cfg)
    Xn, yn = X.numpy(), y.numpy()
    return cfg, X, y, Xn, yn, ridge.closed_form(Xn, yn, cfg.lam)


def test_objective_matches_oracle(rsctx, fp64_problem):
    cfg, X, y, Xn, yn, ws = fp64_problem
    w = ws + 1e-3 * synth.random_vector(cfg.d, 2)
    for dt in (torch.float64, torch.float32):
        L, ex = rs.rs_objective(rsctx, X.to(dt).cuda(), y.to(dt).cuda(), cfg.lam,
                                torch.from_numpy(w).to(dt).cuda(), torch.from_numpy(ws).to(dt).cuda())
        Xd = X.to(dt).double().numpy()
        yd = y.to(dt).double().numpy()
        wd = torch.from_numpy(w).to(dt).double().numpy()
        wsd = torch.from_numpy(ws).to(dt).double().numpy()
        assert L == pytest.approx(ridge.objective(Xd, yd, cfg.lam, wd), rel=1e-12)
        assert ex == pytest.approx(ridge.excess(Xd, cfg.lam, wd, wsd), rel=1e-9)


def test_fp64_alg3_matches_oracle_and_closed_form(rsctx, fp64_problem):
    cfg, X, y, Xn, yn, ws = fp64_problem
    w, info = rs.rs_solve(rsctx, X.cuda(), y.cuda(), cfg.k, cfg.lam, cfg.epochs, cfg.seed_sketch, cfg.seed_svrg,
                          m=cfg.m, eta_mult=cfg.eta_mult, snapshots=True)
    w = w.cpu().numpy()
    rel = ridge.rel_suboptimality(Xn, yn, cfg.lam, w, ws)
    assert rel <= 1e-10, rel
    ref = pipeline.scsvrg(Xn, yn, cfg.lam, cfg.k, cfg.seed_sketch, cfg.seed_svrg, cfg.epochs, m=cfg.m,
                          eta_mult=cfg.eta_mult, history=True)
    assert np.linalg.norm(w - ref["w"]) / np.linalg.norm(ref["w"]) <= 1e-4
    # per-epoch snapshots decrease like the oracle's
    hist = [ridge.rel_suboptimality(Xn, yn, cfg.lam, s, ws) for s in info["snapshots"].cpu().numpy()]
    hist_ref = pipeline.relative_history(Xn, yn, cfg.lam, ref["history"])
    assert hist[-1] <= 1e-10
    for a, b in zip(hist[:8], hist_ref[:8]):
        assert a == pytest.approx(b, rel=0.5)


def test_fp64_trajectory_parity_same_stream(rsctx, fp64_problem):
    """Same data, same preconditioner inputs and same index stream: GPU epochs follow the oracle's
    recursion to rounding (the preconditioner comes from the generator, not from either side)."""
    cfg, X, y, Xn, yn, ws = fp64_problem
    V = synth.random_orthonormal(cfg.d, cfg.k, 5)
    s2 = np.sort(np.linalg.eigvalsh(ridge.correlation(Xn)))[::-1][: cfg.k].copy()
    Z, beta, bh = rs.rs_precondition(rsctx, X.cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(s2).cuda(), cfg.lam)
    M = precond.m_matrix(V, s2, cfg.lam)
    Zr, yz, g = precond.components(*precond.transform(Xn, M), yn, cfg.lam)
    beta_r = precond.smoothness(Zr, g)
    W_gpu = rs.rs_sampling_weights(rsctx, beta).cpu().numpy().view(np.uint32)
    W_ref = streams.quantize_weights(beta_r)
    mism = int(np.sum(W_gpu != W_ref))
    assert mism <= 2, mism
    from oracle import svrg
    w, info = rs.rs_svrg_solve(rsctx, Z, y.cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(s2).cuda(), cfg.lam,
                               3, cfg.seed_svrg, beta=beta, m=2048, eta_mult=1.0)
    snaps = svrg.solve(Zr, yz, g, beta_r, 1.0 / precond.beta_hat(beta_r), 2048, 3, cfg.seed_svrg)
    wr = M @ snaps[-1]
    err = np.linalg.norm(w.cpu().numpy() - wr) / np.linalg.norm(wr)
    assert err <= (1e-10 if mism == 0 else 1e-2), (err, mism)


def test_resume_matches_continuous_run(rsctx, fp64_problem):
    cfg, X, y, Xn, yn, ws = fp64_problem
    V, s2 = rs.rs_sketch(rsctx, X.cuda(), cfg.k, cfg.seed_sketch)
    Z, beta, _ = rs.rs_precondition(rsctx, X.cuda(), V, s2, cfg.lam)
    full, _ = rs.rs_svrg_solve(rsctx, Z, y.cuda(), V, s2, cfg.lam, 4, 9, beta=beta, m=1000, eta_mult=1.0)
    # run 2 epochs, map nothing: take the preconditioned iterate by running with V = identity-free map
    kw = dict(beta=beta, m=1000, eta_mult=1.0)
    part, _ = rs.rs_svrg_solve(rsctx, Z, y.cuda(), V, s2, cfg.lam, 2, 9, **kw)
    # w = M w~: recover w~ = M^{-1} w with the oracle's M (exact inverse in double)
    M = precond.m_matrix(V.cpu().numpy(), s2.cpu().numpy(), cfg.lam)
    wt = np.linalg.solve(M, part.cpu().numpy())
    rest, _ = rs.rs_svrg_solve(rsctx, Z, y.cuda(), V, s2, cfg.lam, 2, 9, w0=torch.from_numpy(wt).cuda(), epoch0=2, **kw)
    np.testing.assert_allclose(rest.cpu().numpy(), full.cpu().numpy(), rtol=1e-9, atol=1e-12)


@pytest.mark.slow
def test_fp32_countsketch_workload_reaches_1e6(rsctx):
    """Full-size FP32 workload (n = 65536, d = 1024, CountSketch s = 4096 then Gaussian k = 64):
    relative suboptimality <= 1e-6 against the double Cholesky solution."""
    cfg = synth.CONFIGS["fp32_n65536_d1024"]
    X, y, _ = synth.config_problem(cfg, device="cuda", dtype=torch.float32)
    Xn = X.double().cpu().numpy()
    yf = y.float()
    ws = ridge.closed_form(Xn, yf.double().cpu().numpy(), cfg.lam)
    w, info = rs.rs_solve(rsctx, X, yf, cfg.k, cfg.lam, 6, cfg.seed_sketch, cfg.seed_svrg, kind="countsketch", s=cfg.s,
                          m=2 * cfg.n, eta_mult=1.0, snapshots=True)
    rel = [ridge.rel_suboptimality(Xn, yf.double().cpu().numpy(), cfg.lam, s.double().cpu().numpy(), ws)
           for s in info["snapshots"]]
    assert rel[-1] <= 1e-6, rel


def test_errors_are_reported(rsctx):
    X = torch.zeros(10, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(rs.RsError) as e:
        rs.rs_sketch(rsctx, X, 9, 0)          # k > d
    assert e.value.code == 1
    with pytest.raises(rs.RsError):
        rs.rs_precondition(rsctx, X, torch.zeros(4, 2, device="cuda"), torch.ones(2, dtype=torch.float64, device="cuda"), -1.0)
    Xo = torch.zeros(10, 5, dtype=torch.float32, device="cuda")   # row stride 20 bytes: not 16-byte aligned
    with pytest.raises(rs.RsError):
        rs.rs_full_gradient(rsctx, Xo[:, :5], torch.zeros(5, device="cuda"), 5, 1e-3, torch.zeros(5, device="cuda"))


@pytest.mark.slow
def test_fp32_workload_trajectory_parity_same_stream(rsctx):
    """Full-size FP32 workload (n = 65536, d = 1024, CountSketch s = 4096 then Gaussian k = 64, lambda =
    1e-5): the GPU's sketch, components and 4 epochs of Alg. 1 (m = 2n, eta = 1/beta^) against the
    oracle replaying the same 4 epochs in float64 from the GPU's V, sigma2 and beta (equal beta gives
    equal integer weights, so both sides draw the same index stream).  The iterates agree to
    ||w - w_oracle|| / ||w_oracle|| <= 1e-4 and both reach relative suboptimality <= 1e-6."""
    from oracle import svrg
    cfg = synth.CONFIGS["fp32_n65536_d1024"]
    X, y64, _ = synth.config_problem(cfg, device="cuda", dtype=torch.float32)
    y = y64.float().contiguous()
    n, d, lam, E, m = cfg.n, cfg.d, cfg.lam, 4, 2 * cfg.n
    V, s2 = rs.rs_sketch(rsctx, X, cfg.k, cfg.seed_sketch, kind=cfg.kind, s=cfg.s)
    Z, beta, _ = rs.rs_precondition(rsctx, X, V, s2, lam)
    w, info = rs.rs_svrg_solve(rsctx, Z, y, V, s2, lam, E, cfg.seed_svrg, beta=beta, m=m, eta_mult=1.0)
    Xn, yn = X.double().cpu().numpy(), y.double().cpu().numpy()
    M = precond.m_matrix(V.double().cpu().numpy(), s2.cpu().numpy(), lam)
    Zr, yz, g = precond.components(*precond.transform(Xn, M), yn, lam)
    snaps = svrg.solve(Zr, yz, g, beta.double().cpu().numpy(), info["eta"], m, E, cfg.seed_svrg)
    wr = M @ snaps[-1]
    wg = w.double().cpu().numpy()
    err = np.linalg.norm(wg - wr) / np.linalg.norm(wr)
    ws = ridge.closed_form(Xn, yn, lam)
    rel_gpu = ridge.rel_suboptimality(Xn, yn, lam, wg, ws)
    rel_orc = ridge.rel_suboptimality(Xn, yn, lam, wr, ws)
    print(f"fp32 workload: |w - w_oracle|/|w_oracle| = {err:.3e}, rel subopt GPU {rel_gpu:.3e}, oracle {rel_orc:.3e}")
    assert err <= 1e-4, err
    assert rel_gpu <= 1e-6 and rel_orc <= 1e-6, (rel_gpu, rel_orc)
