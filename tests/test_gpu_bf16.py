"""BF16 storage with FP32 compute: preconditioned components stored in bfloat16, the full gradient,
the inner loop and Alg. 3 end to end with the refined full gradient (mu formed on the stored data).

The oracle runs in double on the bfloat16 values themselves (the data as stored), so every
comparison measures the FP32 arithmetic plus, where the output is bfloat16, one rounding."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond, ridge, svrg
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu

BF16_UNIT = 2.0 ** -8   # unit roundoff of bfloat16 (8 significand bits)


@pytest.mark.parametrize("n,d,k", [(1, 8, 1), (257, 40, 5), (4096, 256, 16), (65536, 1024, 64), (3000, 520, 70),
                                   (130, 2048, 128), (700, 136, 129)])
@pytest.mark.parametrize("tc", ["1", "0"])
def test_precondition_bf16_matches_oracle(rsctx, monkeypatch, n, d, k, tc):
    """X - P V^T on tensor cores (tcgen05, k <= 128) and on CUDA cores."""
    monkeypatch.setenv("RS_UMMA_RESID", tc)
    X = torch.from_numpy(synth.random_matrix(n, d, n + d, scale=1.0 / np.sqrt(d))).to(torch.bfloat16)
    V = torch.from_numpy(synth.random_orthonormal(d, k, d)).float()
    s2 = synth.random_sigma2(k, k)
    lam = 1e-4
    Z, beta, bh = rs.rs_precondition(rsctx, cuda_rows(X), V.cuda(), torch.from_numpy(s2).cuda(), lam)
    assert Z.dtype == torch.bfloat16 and beta.dtype == torch.float32
    Zg = Z.cpu().double().numpy()
    Xd = X.double().numpy()
    M = precond.m_matrix(V.double().numpy(), s2, lam)
    Xt, B = precond.transform(Xd, M)
    # one bfloat16 rounding of an FP32 result: half an ulp relative, plus the FP32 accumulation
    scale = np.abs(Xd).max() * (1 + np.sqrt(k))
    assert np.all(np.abs(Zg[:n] - Xt) <= BF16_UNIT * np.abs(Xt) + 4e-6 * scale)
    assert np.all(np.abs(Zg[n:] - B) <= BF16_UNIT * np.abs(B) + 4e-6 * (1 + np.sqrt(k)))
    # beta comes from the stored (rounded) rows: compare with the oracle on those rows
    _, _, g = precond.components(Zg[:n], Zg[n:], np.zeros(n), lam)
    beta_ref = precond.smoothness(Zg, g)
    np.testing.assert_allclose(beta.cpu().double().numpy(), beta_ref, rtol=2e-5 * np.sqrt(d))
    assert bh == pytest.approx(precond.beta_hat(beta_ref), rel=2e-5 * np.sqrt(d))


def _bf16_components(n, d, seed, lam):
    Z = torch.from_numpy(synth.random_matrix(n + d, d, seed, scale=1.0 / np.sqrt(d))).to(torch.bfloat16)
    y = torch.from_numpy(synth.random_vector(n, seed + 1)).float()
    Zd = Z.double().numpy()
    _, yz, g = precond.components(Zd[:n], Zd[n:], y.double().numpy(), lam)
    return cuda_rows(Z), Zd, y.cuda(), yz, g


@pytest.mark.parametrize("n,d", [(1, 8), (5000, 40), (4096, 256), (3000, 520), (65536, 1024), (20000, 2056)])
def test_full_gradient_bf16_matches_oracle(rsctx, n, d):
    lam = 1e-3
    Z, Zd, y, yz, g = _bf16_components(n, d, n + d, lam)
    w = torch.from_numpy(synth.random_vector(d, 1)).float()
    mu = rs.rs_full_gradient(rsctx, Z, y, n, lam, w.cuda()).cpu().double().numpy()
    ref = svrg.full_gradient_fast(Zd, yz, g, w.double().numpy())
    scale = np.abs(Zd).max() * np.abs(g * (Zd @ w.double().numpy() - yz)).mean() * 4
    np.testing.assert_allclose(mu, ref, rtol=0, atol=1e-5 * max(scale, np.abs(ref).max()))


@pytest.mark.parametrize("n,d,m", [(50, 8, 1), (300, 64, 65), (2000, 256, 1000), (3000, 104, 777), (700, 100, 300),
                                   (40, 3, 70), (8000, 1024, 4160), (4000, 2048, 640)])
@pytest.mark.parametrize("average", [True, False])
@pytest.mark.parametrize("tc_prep", ["1", "0"])
def test_epoch_bf16_matches_stepwise_oracle(rsctx, monkeypatch, n, d, m, average, tc_prep):
    """Both block preparations: tensor-core Gram matrices (tcgen05) and the CUDA-core kernel."""
    monkeypatch.setenv("RS_UMMA_PREP", tc_prep)
    lam = 1e-3
    Z, Zd, y, yz, g = _bf16_components(n, d, 7 * n + d, lam)
    N = n + d
    idx = synth.random_indices(N, m, m + d)
    inq = torch.from_numpy(synth.random_positive(m, m, 0.5, 1.5)).float()
    beta = precond.smoothness(Zd, g)
    eta = 0.2 / beta.mean()
    w_bar = torch.from_numpy(synth.random_vector(d, 5, scale=0.1)).float()
    mu = torch.from_numpy(synth.random_vector(d, 6, scale=1e-3)).float()
    got = rs.rs_svrg_epoch(rsctx, Z, n, lam, torch.from_numpy(idx.astype(np.int32)).cuda(), inq.cuda(), eta,
                           w_bar.cuda(), mu.cuda(), average).cpu().double().numpy()
    ref = svrg.epoch_scaled(Zd, yz, g, w_bar.double().numpy(), idx, inq.double().numpy(), eta, average,
                            v_bar=mu.double().numpy())
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err


@pytest.fixture(scope="module")
def bf16_problem():
    n, d, k, lam = 8192, 256, 16, 1e-4
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.5, 0.1, 77)
    Xb = X.to(torch.bfloat16)
    Xd = Xb.double().numpy()
    yf = y.float()
    ws = ridge.closed_form(Xd, yf.double().numpy(), lam)
    return n, d, k, lam, Xb, yf, Xd, ws


def test_bf16_alg3_with_refinement_reaches_fp32_accuracy(rsctx, bf16_problem):
    """Alg. 3 on BF16 data: with the refined full gradient the iterate converges to the minimiser of
    Eq. (1) for the data as stored, to FP32 accuracy (relative suboptimality <= 1e-8)."""
    n, d, k, lam, Xb, yf, Xd, ws = bf16_problem
    w, info = rs.rs_solve(rsctx, cuda_rows(Xb), yf.cuda(), k, lam, 14, 11, 12, m=2 * n, eta_mult=1.0,
                          refine=True, snapshots=True)
    rel = [ridge.rel_suboptimality(Xd, yf.double().numpy(), lam, s.double().cpu().numpy(), ws)
           for s in info["snapshots"]]
    assert rel[-1] <= 1e-8, rel
    # converges linearly: the last epochs improve on the first by orders of magnitude
    assert rel[-1] <= 1e-3 * rel[0], rel


def test_bf16_refinement_beats_plain_components(rsctx, bf16_problem):
    """Without refinement the fixed point is that of the rounded components; it stalls above the
    refined run (the rounding of Z perturbs the problem by about 2^-9 per entry)."""
    n, d, k, lam, Xb, yf, Xd, ws = bf16_problem
    yn = yf.double().numpy()
    w_r, _ = rs.rs_solve(rsctx, cuda_rows(Xb), yf.cuda(), k, lam, 14, 11, 12, m=2 * n, eta_mult=1.0, refine=True)
    w_p, _ = rs.rs_solve(rsctx, cuda_rows(Xb), yf.cuda(), k, lam, 14, 11, 12, m=2 * n, eta_mult=1.0, refine=False)
    r_ref = ridge.rel_suboptimality(Xd, yn, lam, w_r.double().cpu().numpy(), ws)
    r_pl = ridge.rel_suboptimality(Xd, yn, lam, w_p.double().cpu().numpy(), ws)
    assert np.isfinite(r_pl) and r_ref <= r_pl, (r_ref, r_pl)


def test_bf16_svrg_solve_requires_data_for_refinement(rsctx, bf16_problem):
    n, d, k, lam, Xb, yf, Xd, ws = bf16_problem
    Xc = cuda_rows(Xb)
    V, s2 = rs.rs_sketch(rsctx, Xc, k, 3)
    Z, beta, _ = rs.rs_precondition(rsctx, Xc, V, s2, lam)
    with pytest.raises(rs.RsError):
        rs.rs_svrg_solve(rsctx, Z, yf.cuda(), V, s2, lam, 1, 5, beta=beta, refine=True)   # X missing
    w, _ = rs.rs_svrg_solve(rsctx, Z, yf.cuda(), V, s2, lam, 2, 5, beta=beta, refine=True, X=Xc, m=n)
    assert torch.isfinite(w).all()


@pytest.mark.parametrize("n,d,k", [(257, 40, 5), (3000, 520, 60), (65536, 1024, 64), (2000, 256, 100)])
@pytest.mark.parametrize("tc", ["1", "0"])
def test_bf16_components_from_float_data(rsctx, monkeypatch, n, d, k, tc):
    """Float data, bfloat16 components: each z_i is formed in float and rounded once (tensor-core
    path from the bfloat16 parts of X for k <= 64, and CUDA cores)."""
    monkeypatch.setenv("RS_UMMA", tc)
    X = torch.from_numpy(synth.random_matrix(n, d, n + 2 * d, scale=1.0 / np.sqrt(d))).float()
    V = torch.from_numpy(synth.random_orthonormal(d, k, d + 1)).float()
    s2 = synth.random_sigma2(k, k + 1)
    lam = 1e-4
    Z, beta, bh = rs.rs_precondition(rsctx, cuda_rows(X), V.cuda(), torch.from_numpy(s2).cuda(), lam,
                                     z_dtype=torch.bfloat16)
    assert Z.dtype == torch.bfloat16
    Zg = Z.cpu().double().numpy()
    M = precond.m_matrix(V.double().numpy(), s2, lam)
    Xt, B = precond.transform(X.double().numpy(), M)
    scale = np.abs(X.double().numpy()).max() * (1 + np.sqrt(k))
    assert np.all(np.abs(Zg[:n] - Xt) <= BF16_UNIT * np.abs(Xt) + 4e-6 * scale)
    assert np.all(np.abs(Zg[n:] - B) <= BF16_UNIT * np.abs(B) + 4e-6 * (1 + np.sqrt(k)))


def test_bf16_components_with_float_refinement_reach_float_accuracy(rsctx):
    """BF16 components and the refined gradient on the float data: the iterate converges to the
    minimiser of Eq. (1) for the float data itself."""
    n, d, k, lam = 8192, 256, 16, 1e-4
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1, dtype=np.float64) ** -1.5, 0.1, 78)
    Xf, yf = X.float(), y.float()
    Xd, yn = Xf.double().numpy(), yf.double().numpy()
    ws = ridge.closed_form(Xd, yn, lam)
    Xc = cuda_rows(Xf)
    V, s2 = rs.rs_sketch(rsctx, Xc, k, 3)
    Z, beta, _ = rs.rs_precondition(rsctx, Xc, V, s2, lam, z_dtype=torch.bfloat16)
    w, info = rs.rs_svrg_solve(rsctx, Z, yf.cuda(), V, s2, lam, 14, 5, beta=beta, m=2 * n, eta_mult=1.0, X=Xc,
                               refine=True, snapshots=True)
    rel = [ridge.rel_suboptimality(Xd, yn, lam, s.double().cpu().numpy(), ws) for s in info["snapshots"]]
    assert rel[-1] <= 1e-8, rel


@pytest.mark.parametrize("umma", ["1", "0"])
@pytest.mark.parametrize("n,d,k", [(1, 8, 1), (300, 72, 5), (4097, 256, 16), (20000, 1024, 130)])
def test_bf16_x_times_v_both_paths(rsctx, monkeypatch, umma, n, d, k):
    """X V for bfloat16 data on the tensor cores (tcgen05, V split into three bfloat16 parts) and
    on CUDA cores give the oracle's components to the same tolerance."""
    monkeypatch.setenv("RS_UMMA", umma)
    monkeypatch.setenv("RS_UMMA_RESID", umma)
    X = torch.from_numpy(synth.random_matrix(n, d, 3 * n + d, scale=1.0 / np.sqrt(d))).to(torch.bfloat16)
    V = torch.from_numpy(synth.random_orthonormal(d, k, d + 5)).float()
    s2 = synth.random_sigma2(k, k + 3)
    lam = 1e-4
    Z, beta, bh = rs.rs_precondition(rsctx, cuda_rows(X), V.cuda(), torch.from_numpy(s2).cuda(), lam)
    Zg = Z.cpu().double().numpy()
    M = precond.m_matrix(V.double().numpy(), s2, lam)
    Xt, B = precond.transform(X.double().numpy(), M)
    scale = np.abs(X.double().numpy()).max() * (1 + np.sqrt(k))
    assert np.all(np.abs(Zg[:n] - Xt) <= BF16_UNIT * np.abs(Xt) + 4e-6 * scale)


@pytest.mark.parametrize("umma", ["1", "0"])
@pytest.mark.parametrize("n,d,k", [(1, 8, 1), (300, 72, 5), (4097, 256, 16), (20000, 1024, 130), (65536, 1024, 64)])
def test_f32_x_times_v_both_paths(rsctx, monkeypatch, umma, n, d, k):
    """X V and X Q for float data on the tensor cores (X and W each split into three bfloat16
    parts, six products) and on CUDA cores: float components to FP32 accuracy, and the
    Rayleigh-Ritz step (Alg. 2) on the same data."""
    monkeypatch.setenv("RS_UMMA", umma)
    X = torch.from_numpy(synth.random_matrix(n, d, 5 * n + d, scale=1.0 / np.sqrt(d))).float()
    V = torch.from_numpy(synth.random_orthonormal(d, k, d + 7)).float()
    s2 = synth.random_sigma2(k, k + 1)
    lam = 1e-4
    Z, _, _ = rs.rs_precondition(rsctx, cuda_rows(X), V.cuda(), torch.from_numpy(s2).cuda(), lam)
    Zg = Z.cpu().double().numpy()
    M = precond.m_matrix(V.double().numpy(), s2, lam)
    Xt, _ = precond.transform(X.double().numpy(), M)
    scale = np.abs(X.double().numpy()).max() * (1 + np.sqrt(k))
    np.testing.assert_allclose(Zg[:n], Xt, rtol=0, atol=2e-6 * scale)
