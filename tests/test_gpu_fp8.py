"""FP8-e4m3 component storage with one scale per row (value = code * scale), float arithmetic, and
snapshot gradients refined on the float data.  The oracle runs on the dequantised values (the
data the inner loop actually sees) and, end to end, on the float data itself."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond, ridge, svrg
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu

E4M3_HALF_ULP = 2.0 ** -4     # 3 explicit mantissa bits: half an ulp relative
E4M3_MIN_SUB = 2.0 ** -9      # smallest subnormal step of e4m3 (relative to the row scale)


@pytest.mark.parametrize("xdt", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("n,d,k", [(1, 16, 1), (300, 48, 5), (8192, 256, 16)])
def test_precondition_fp8_rows(rsctx, xdt, n, d, k):
    X = torch.from_numpy(synth.random_matrix(n, d, n + 5 * d, scale=1.0 / np.sqrt(d))).to(xdt)
    V = torch.from_numpy(synth.random_orthonormal(d, k, d + 9)).float()
    s2 = synth.random_sigma2(k, k + 7)
    lam = 1e-4
    Z, beta, bh = rs.rs_precondition(rsctx, cuda_rows(X), V.cuda(), torch.from_numpy(s2).cuda(), lam,
                                     z_dtype=torch.float8_e4m3fn)
    sc = Z.scale.cpu().double().numpy()
    deq = Z.dequantize().cpu().double().numpy()
    M = precond.m_matrix(V.double().numpy(), s2, lam)
    Xt, B = precond.transform(X.double().numpy(), M)
    ref = np.vstack([Xt, B])
    # every row's largest code is 448 at most, and the scale is the row maximum / 448 (via bfloat16)
    rowmax = np.abs(ref).max(1)
    np.testing.assert_allclose(sc * 448.0, rowmax, rtol=2 * 2.0 ** -8)
    # one e4m3 rounding (plus the bfloat16 staging rounding) per element
    bound = (E4M3_HALF_ULP + 2.0 ** -8) * np.abs(ref) + E4M3_MIN_SUB * sc[:, None] + 1e-6
    assert np.all(np.abs(deq - ref) <= bound)
    # beta from the stored values
    _, _, g = precond.components(deq[:n], deq[n:], np.zeros(n), lam)
    np.testing.assert_allclose(beta.cpu().double().numpy(), precond.smoothness(deq, g), rtol=1e-5)


@pytest.mark.parametrize("n,d,m", [(300, 64, 65), (2000, 256, 1000), (4000, 1024, 2050), (3000, 104, 777)])
def test_epoch_fp8_matches_stepwise_oracle(rsctx, n, d, m):
    """The inner loop on FP8 codes with row scales follows the oracle's recursion on the
    dequantised rows."""
    lam = 1e-3
    Zf = synth.random_matrix(n + d, d, 5 * n + d, scale=1.0 / np.sqrt(d))
    codes_ld = (d + 15) // 16 * 16
    sc = np.abs(Zf).max(1) / 448.0
    q = torch.zeros(n + d, codes_ld, dtype=torch.float8_e4m3fn)
    q[:, :d] = torch.from_numpy(Zf / sc[:, None]).float().to(torch.float8_e4m3fn)
    Z = rs.Fp8Rows(q.cuda()[:, :d], torch.from_numpy(sc).float().cuda())
    Zd = q[:, :d].double().numpy() * torch.from_numpy(sc).float().double().numpy()[:, None]
    y = synth.random_vector(n, 7)
    _, yz, g = precond.components(Zd[:n], Zd[n:], y, lam)
    N = n + d
    idx = synth.random_indices(N, m, m + 11)
    inq = torch.from_numpy(synth.random_positive(m, m + 2, 0.5, 1.5)).float()
    beta = precond.smoothness(Zd, g)
    eta = 0.2 / beta.mean()
    w_bar = torch.from_numpy(synth.random_vector(d, 5, scale=0.1)).float()
    mu = torch.from_numpy(synth.random_vector(d, 6, scale=1e-3)).float()
    got = rs.rs_svrg_epoch(rsctx, Z, n, lam, torch.from_numpy(idx.astype(np.int32)).cuda(), inq.cuda(), eta,
                           w_bar.cuda(), mu.cuda(), True).cpu().double().numpy()
    ref = svrg.epoch_scaled(Zd, yz, g, w_bar.double().numpy(), idx, inq.double().numpy(), eta, True,
                            v_bar=mu.double().numpy())
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4


def test_fp8_components_with_refinement_converge(rsctx):
    """FP8 components, snapshot gradients on the float data: the iterate converges to the minimiser
    of Eq. (1) for the float data (the rounding of the components slows it, it does not bias it)."""
    n, d, k, lam = 8192, 256, 16, 1e-4
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.5, 0.1, 79)
    Xf, yf = X.float(), y.float()
    Xd, yn = Xf.double().numpy(), yf.double().numpy()
    ws = ridge.closed_form(Xd, yn, lam)
    Xc = cuda_rows(Xf)
    V, s2 = rs.rs_sketch(rsctx, Xc, k, 3)
    Z, beta, _ = rs.rs_precondition(rsctx, Xc, V, s2, lam, z_dtype=torch.float8_e4m3fn)
    w, info = rs.rs_svrg_solve(rsctx, Z, yf.cuda(), V, s2, lam, 30, 5, beta=beta, m=n, eta_mult=0.5, X=Xc,
                               refine=True, snapshots=True)
    rel = [ridge.rel_suboptimality(Xd, yn, lam, s.double().cpu().numpy(), ws) for s in info["snapshots"]]
    assert rel[-1] <= 1e-6, rel
    assert rel[-1] <= 1e-3 * rel[0]


def test_fp8_solve_requires_refinement(rsctx):
    n, d = 512, 32
    X = cuda_rows(torch.from_numpy(synth.random_matrix(n, d, 3)).float())
    V, s2 = rs.rs_sketch(rsctx, X, 4, 1)
    Z, beta, _ = rs.rs_precondition(rsctx, X, V, s2, 1e-3, z_dtype=torch.float8_e4m3fn)
    with pytest.raises(rs.RsError):
        rs.rs_svrg_solve(rsctx, Z, torch.zeros(n, device="cuda"), V, s2, 1e-3, 1, 1, beta=beta)
