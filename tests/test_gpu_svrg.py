"""GPU parity of SVRG (Alg. 1): the full-gradient pass and the blocked inner loop, replayed on the
same generator index streams and weights as the oracle's step-by-step recursion."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond, svrg
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


def _components(n, d, seed, dtype, lam):
    """Generator rows for the N = n + d components (rows scaled to norm ~1) and labels."""
    Z = synth.random_matrix(n + d, d, seed, scale=1.0 / np.sqrt(d))
    y = synth.random_vector(n, seed + 1)
    Zt = torch.from_numpy(Z).to(dtype)
    ld = ((d * Zt.element_size() + 15) // 16 * 16) // Zt.element_size()
    buf = torch.zeros(n + d, ld, dtype=dtype)
    buf[:, :d] = Zt
    Zd = buf[:, :d].double().numpy()
    _, yz, g = precond.components(Zd[:n], Zd[n:], y, lam)
    return buf.cuda()[:, :d], Zd, torch.from_numpy(y).to(dtype).cuda(), yz, g


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("n,d", [(1, 3), (5000, 37), (4096, 256), (3000, 513), (65536, 1024), (20000, 2050)])
def test_full_gradient_matches_oracle(rsctx, dtype, tol, n, d):
    lam = 1e-3
    Z, Zd, y, yz, g = _components(n, d, n + d, dtype, lam)
    w = synth.random_vector(d, 1)
    wt = torch.from_numpy(w).to(dtype)
    mu = rs.rs_full_gradient(rsctx, Z, y, n, lam, wt.cuda()).cpu().double().numpy()
    ref = svrg.full_gradient_fast(Zd, yz, g, wt.double().numpy())
    # each component of mu sums N terms of size ~|r| |z|: compare against that scale
    scale = np.abs(Zd).max() * np.abs(g * (Zd @ wt.double().numpy() - yz)).mean() * 4
    np.testing.assert_allclose(mu, ref, rtol=0, atol=tol * max(scale, np.abs(ref).max()))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 1e-4)])
@pytest.mark.parametrize("n,d,m", [(50, 7, 1), (300, 64, 63), (300, 64, 64), (300, 64, 65), (2000, 256, 1000),
                                   (4096, 256, 8192), (8000, 1024, 4160), (3000, 100, 777)])
@pytest.mark.parametrize("average", [True, False])
def test_epoch_matches_stepwise_oracle(rsctx, dtype, tol, n, d, m, average):
    if dtype == torch.float64 and d > 256:
        pytest.skip("covered in float")
    lam = 1e-3
    Z, Zd, y, yz, g = _components(n, d, 7 * n + d, dtype, lam)
    N = n + d
    idx = synth.random_indices(N, m, m + d)
    inq = synth.random_positive(m, m, 0.5, 1.5)
    inq_t = torch.from_numpy(inq).to(dtype)
    inq_d = inq_t.double().numpy()
    beta = precond.smoothness(Zd, g)
    eta = 0.2 / beta.mean()
    w_bar = synth.random_vector(d, 5, scale=0.1)
    mu = synth.random_vector(d, 6, scale=1e-3)
    wb_t = torch.from_numpy(w_bar).to(dtype)
    mu_t = torch.from_numpy(mu).to(dtype)
    got = rs.rs_svrg_epoch(rsctx, Z, n, lam, torch.from_numpy(idx.astype(np.int32)).cuda(), inq_t.cuda(), eta,
                           wb_t.cuda(), mu_t.cuda(), average).cpu().double().numpy()
    ref = svrg.epoch_scaled(Zd, yz, g, wb_t.double().numpy(), idx, inq_d, eta, average, v_bar=mu_t.double().numpy())
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err


def test_epoch_rejects_bad_arguments(rsctx):
    Z, _, y, _, _ = _components(20, 4, 1, torch.float32, 1e-3)
    w = torch.zeros(4, device="cuda")
    idx = torch.zeros(3, dtype=torch.int32, device="cuda")
    inq = torch.ones(3, device="cuda")
    with pytest.raises(rs.RsError):
        rs._lib._check(rs.lib().rs_svrg_epoch(rsctx.h, rs._lib.ctypes.byref(rs.matrix(Z)), 20, 1e-3,
                                              rs._lib._ptr(idx), rs._lib._ptr(inq), 3, 0.1, rs._lib._ptr(w),
                                              rs._lib._ptr(w), 1, rs._lib._ptr(w)))
    with pytest.raises(rs.RsError):
        rs.rs_full_gradient(rsctx, Z, y, 25, 1e-3, w)     # n + d != rows


@pytest.mark.parametrize("lookahead", ["0", "1"])
@pytest.mark.parametrize("n,d,m", [(300, 64, 65), (2000, 256, 1000), (8000, 1024, 4160), (3000, 520, 129)])
def test_epoch_both_chain_variants(rsctx, monkeypatch, lookahead, n, d, m):
    """The plain chain (exchange on the critical path) and the look-ahead chain (next block's dots
    exchanged while the current block updates) both follow the oracle's recursion."""
    monkeypatch.setenv("RS_CHAIN_LOOKAHEAD", lookahead)
    lam = 1e-3
    Z, Zd, y, yz, g = _components(n, d, 11 * n + d, torch.float32, lam)
    N = n + d
    idx = synth.random_indices(N, m, m + 3 * d)
    inq_t = torch.from_numpy(synth.random_positive(m, m + 1, 0.5, 1.5)).float()
    beta = precond.smoothness(Zd, g)
    eta = 0.3 / beta.mean()
    wb_t = torch.from_numpy(synth.random_vector(d, 7, scale=0.1)).float()
    mu_t = torch.from_numpy(synth.random_vector(d, 8, scale=1e-3)).float()
    got = rs.rs_svrg_epoch(rsctx, Z, n, lam, torch.from_numpy(idx.astype(np.int32)).cuda(), inq_t.cuda(), eta,
                           wb_t.cuda(), mu_t.cuda(), True).cpu().double().numpy()
    ref = svrg.epoch_scaled(Zd, yz, g, wb_t.double().numpy(), idx, inq_t.double().numpy(), eta, True,
                            v_bar=mu_t.double().numpy())
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
