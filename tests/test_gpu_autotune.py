"""The autotuner (rs_autotune): it times the launch layouts of the inner loop and the full-gradient
pass, keeps the fastest per (storage type, width) in the context, answers a repeated call from the
cache, and the tuned layouts compute the same results (the oracle's step-by-step loop for the inner
loop; the untuned context for both)."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond, svrg
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


def _components(n, d, seed, dtype, lam):
    Z = synth.random_matrix(n + d, d, seed, scale=1.0 / np.sqrt(d))
    y = synth.random_vector(n, seed + 1)
    Zt = torch.from_numpy(Z).to(dtype)
    Zd = Zt.double().numpy()
    _, yz, g = precond.components(Zd[:n], Zd[n:], y, lam)
    return Zt.cuda(), Zd, torch.from_numpy(y).float().cuda(), yz, g


@pytest.mark.parametrize("dtype,n,d", [(torch.float32, 8000, 1024), (torch.bfloat16, 6000, 4096),
                                       (torch.float32, 3000, 520)])
def test_autotune_chooses_a_valid_layout_and_caches_it(dtype, n, d):
    lam = 1e-3
    Z, Zd, y, yz, g = _components(n, d, n + d, dtype, lam)
    with rs.Context(0) as ctx:
        rep = rs.rs_autotune(ctx, Z, n)
        cs = rep["chain_cluster"]
        assert cs in (1, 2, 4, 8, 16) and (d + cs - 1) // cs <= 256
        assert rep["chain_threads"] in (256, 512) and rep["chain_stages"] in (2, 3, 4)
        assert rep["chain_ms"] > 0 and rep["candidates"] >= 2 and rep["cached"] == 0
        assert rep["fullgrad_stages"] in (2, 3, 4, 6, 8) and rep["fullgrad_ms"] > 0
        again = rs.rs_autotune(ctx, Z, n)
        assert again["cached"] == 1 and again["candidates"] == 0
        for key in ("chain_cluster", "chain_threads", "chain_stages", "fullgrad_stages"):
            assert again[key] == rep[key]
        # the tuned layouts give the same full gradient and epoch as an untuned context
        m = 2000
        idx = torch.from_numpy(synth.random_indices(n + d, m, 5).astype(np.int32)).cuda()
        inq = torch.from_numpy(synth.random_positive(m, 6, 0.5, 1.5)).float().cuda()
        eta = 0.2 / precond.smoothness(Zd, g).mean()
        wb = torch.from_numpy(synth.random_vector(d, 7, scale=0.1)).float().cuda()
        mu_t = rs.rs_full_gradient(ctx, Z, y, n, lam, wb)
        got = rs.rs_svrg_epoch(ctx, Z, n, lam, idx, inq, eta, wb, mu_t * 1e-3, True).double().cpu().numpy()
    with rs.Context(0) as ctx2:
        mu_d = rs.rs_full_gradient(ctx2, Z, y, n, lam, wb)
        dflt = rs.rs_svrg_epoch(ctx2, Z, n, lam, idx, inq, eta, wb, mu_t * 1e-3, True).double().cpu().numpy()
    scale = float(mu_d.abs().max())
    assert float((mu_t - mu_d).abs().max()) <= 1e-5 * scale
    assert np.linalg.norm(got - dflt) / np.linalg.norm(dflt) <= 1e-5
    ref = svrg.epoch_scaled(Zd, yz, g, wb.double().cpu().numpy(), idx.cpu().numpy(), inq.double().cpu().numpy(), eta,
                            True, v_bar=(mu_t * 1e-3).double().cpu().numpy())
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
