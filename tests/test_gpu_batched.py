"""Batched solves (many problems x lambda path x SVRG settings in batched launches and one CUDA
graph): agreement with the one-chain path on the same sketch, components and index streams,
convergence to the closed-form minimiser of each (problem, lambda), graph vs eager execution."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import ridge
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu


def _problem(n, d, alpha, seed, dtype=torch.float32):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -alpha, 0.05, seed)
    Xs = X.to(dtype)
    return cuda_rows(Xs), y.float().cuda(), Xs.double().numpy(), y.float().double().numpy()


@pytest.fixture(scope="module")
def small_batch():
    probs = [_problem(3000, 64, 1.5, 1), _problem(2000, 128, 2.0, 2), _problem(5000, 64, 1.2, 3)]
    return probs


@pytest.mark.parametrize("refine", [False, True])
def test_batched_matches_single_chain_path(rsctx, small_batch, refine):
    probs = small_batch
    k = 8
    chains = []
    for p in range(len(probs)):
        for lam in (1e-3, 1e-4):
            chains.append(dict(problem=p, lam=lam, eta_mult=1.0, m=probs[p][0].shape[0], seed=100 + p))
    chains.append(dict(problem=1, lam=1e-3, eta_mult=0.5, m=1000, seed=7))
    epochs = 4
    ws, _, _ = rs.rs_solve_batched(rsctx, [(X, y, k) for X, y, _, _ in probs], chains, epochs, sketch_seed=50,
                                   refine=refine)
    for ch, w in zip(chains, ws):
        X, y, _, _ = probs[ch["problem"]]
        V, s2 = rs.rs_sketch(rsctx, X, k, 50 + ch["problem"])
        Z, beta, _ = rs.rs_precondition(rsctx, X, V, s2, ch["lam"])
        w1, _ = rs.rs_svrg_solve(rsctx, Z, y, V, s2, ch["lam"], epochs, ch["seed"], beta=beta, m=ch["m"],
                                 eta_mult=ch["eta_mult"], X=X if refine else None, refine=refine)
        err = (w - w1).norm().item() / w1.norm().item()
        assert err <= 1e-4, (ch, err)


def test_batched_lambda_path_converges(rsctx, small_batch):
    probs = small_batch
    lams = [1e-2, 3e-3, 1e-3]
    chains = [dict(problem=p, lam=lam, eta_mult=1.0, m=probs[p][0].shape[0] // 2, seed=p)
              for p in range(len(probs)) for lam in lams]
    epochs = 30
    ws, snaps, ems = rs.rs_solve_batched(rsctx, [(X, y, 32) for X, y, _, _ in probs], chains, epochs,
                                         sketch_seed=9, snapshots=True)
    assert len(ems) == epochs and all(np.diff(ems) >= 0)
    for ch, w, sn in zip(chains, ws, snaps):
        _, _, Xd, yd = probs[ch["problem"]]
        ws_ = ridge.closed_form(Xd, yd, ch["lam"])
        rel = ridge.rel_suboptimality(Xd, yd, ch["lam"], w.double().cpu().numpy(), ws_)
        assert rel <= 1e-6, (ch, rel)
        np.testing.assert_array_equal(sn[-1].cpu().numpy(), w.cpu().numpy())


def test_batched_bf16_with_refinement(rsctx):
    probs = [_problem(4000, 256, 1.5, 11, torch.bfloat16), _problem(3000, 512, 2.0, 12, torch.bfloat16)]
    chains = [dict(problem=p, lam=lam, eta_mult=1.0, m=probs[p][0].shape[0] // 2, seed=3)
              for p in range(2) for lam in (1e-2, 1e-3)]
    ws, _, _ = rs.rs_solve_batched(rsctx, [(X, y, 0) for X, y, _, _ in probs], chains, 30, sketch_seed=4)
    for ch, w in zip(chains, ws):
        _, _, Xd, yd = probs[ch["problem"]]
        ws_ = ridge.closed_form(Xd, yd, ch["lam"])
        rel = ridge.rel_suboptimality(Xd, yd, ch["lam"], w.double().cpu().numpy(), ws_)
        assert rel <= 1e-6, (ch, rel)


def test_graph_and_eager_agree_bitwise(rsctx, small_batch):
    probs = small_batch
    chains = [dict(problem=p, lam=1e-3, m=700, seed=p) for p in range(len(probs))]
    args = ([(X, y, 8) for X, y, _, _ in probs], chains, 5)
    wg, _, _ = rs.rs_solve_batched(rsctx, *args, sketch_seed=1, use_graph=True)
    we, _, _ = rs.rs_solve_batched(rsctx, *args, sketch_seed=1, use_graph=False)
    for a, b in zip(wg, we):
        assert torch.equal(a, b)


def test_batched_mixed_widths(rsctx):
    """Problems of d = 256, 512, 1024 and 2048 in one call (four inner-loop launches per epoch)."""
    probs = [_problem(2048 + 512 * i, d, 1.0 + 0.3 * i, 20 + i) for i, d in enumerate([256, 2048, 512, 1024])]
    chains = [dict(problem=p, lam=1e-3, eta_mult=1.0, m=1024, seed=p) for p in range(4)]
    ws, _, _ = rs.rs_solve_batched(rsctx, [(X, y, 0) for X, y, _, _ in probs], chains, 3, sketch_seed=2)
    for ch, w in zip(chains, ws):
        X, y, _, _ = probs[ch["problem"]]
        k = max(1, X.shape[1] // 16)
        V, s2 = rs.rs_sketch(rsctx, X, k, 2 + ch["problem"])
        Z, beta, _ = rs.rs_precondition(rsctx, X, V, s2, 1e-3)
        w1, _ = rs.rs_svrg_solve(rsctx, Z, y, V, s2, 1e-3, 3, ch["seed"], beta=beta, m=1024, eta_mult=1.0)
        assert (w - w1).norm().item() <= 1e-4 * w1.norm().item()


def test_batched_rejects_bad_input(rsctx, small_batch):
    X, y, _, _ = small_batch[0]
    with pytest.raises(rs.RsError):
        rs.rs_solve_batched(rsctx, [(X, y, 8)], [dict(problem=1, lam=1e-3)], 2)
    with pytest.raises(rs.RsError):
        rs.rs_solve_batched(rsctx, [(X, y, 8)], [dict(problem=0, lam=-1.0)], 2)
    Xb = cuda_rows(torch.zeros(100, 16, dtype=torch.bfloat16))
    with pytest.raises(rs.RsError):
        rs.rs_solve_batched(rsctx, [(Xb, torch.zeros(100, device="cuda"), 2)], [dict(problem=0, lam=1e-3)], 2,
                            refine=False)


@pytest.mark.parametrize("nchains", [12, 20])
def test_batched_many_chains_per_problem(rsctx, nchains):
    """More than 8 chains on one problem (the refined-gradient passes run with 16 or 32 columns):
    every chain agrees with the one-chain path on the same sketch, components and streams."""
    X, y, _, _ = _problem(3000, 256, 1.5, 41, torch.bfloat16)
    lams = [10.0 ** (-2 - 2 * j / (nchains - 1)) for j in range(nchains)]
    chains = [dict(problem=0, lam=lam, eta_mult=1.0, m=1500, seed=j) for j, lam in enumerate(lams)]
    epochs = 3
    ws, _, _ = rs.rs_solve_batched(rsctx, [(X, y, 16)], chains, epochs, sketch_seed=5)
    V, s2 = rs.rs_sketch(rsctx, X, 16, 5)
    for ch, w in zip(chains[:: max(1, nchains // 4)], ws[:: max(1, nchains // 4)]):
        Z, beta, _ = rs.rs_precondition(rsctx, X, V, s2, ch["lam"])
        w1, _ = rs.rs_svrg_solve(rsctx, Z, y, V, s2, ch["lam"], epochs, ch["seed"], beta=beta, m=ch["m"],
                                 eta_mult=1.0, X=X, refine=True)
        err = (w - w1).norm().item() / w1.norm().item()
        assert err <= 1e-4, (ch, err)


def test_batched_chains_follow_the_oracle(rsctx, small_batch):
    """Every chain of a batched call against the oracle's Alg. 1 replayed in float64 on the same
    components (from the same sketch seed), smoothness constants (so the same integer weights and
    index stream), step size and epoch length: ||w - w_oracle|| / ||w_oracle|| <= 1e-4 (FP32)."""
    from oracle import precond, svrg
    probs = small_batch
    k, epochs = 8, 3
    chains = [dict(problem=p, lam=lam, eta_mult=1.0, m=probs[p][0].shape[0], seed=200 + p)
              for p in range(len(probs)) for lam in (1e-3, 3e-5)]
    ws, _, _ = rs.rs_solve_batched(rsctx, [(X, y, k) for X, y, _, _ in probs], chains, epochs, sketch_seed=60,
                                   refine=False)
    for ch, w in zip(chains, ws):
        X, y, Xn, yn = probs[ch["problem"]]
        n = Xn.shape[0]
        lam = ch["lam"]
        V, s2 = rs.rs_sketch(rsctx, X, k, 60 + ch["problem"])
        _, beta, _ = rs.rs_precondition(rsctx, X, V, s2, lam)
        M = precond.m_matrix(V.double().cpu().numpy(), s2.cpu().numpy(), lam)
        Zr, yz, g = precond.components(*precond.transform(Xn, M), yn, lam)
        b = beta.double().cpu().numpy()
        snaps = svrg.solve(Zr, yz, g, b, ch["eta_mult"] / precond.beta_hat(b), ch["m"], epochs, ch["seed"])
        wr = M @ snaps[-1]
        err = np.linalg.norm(w.double().cpu().numpy() - wr) / np.linalg.norm(wr)
        assert err <= 1e-4, (ch, err)
