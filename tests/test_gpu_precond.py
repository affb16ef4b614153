"""GPU parity of the preconditioner (Eq. (11), Sec. 5.1): transformed rows, regulariser rows,
smoothness constants and the output map, against the oracle on generator inputs."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("n,d,k", [(1, 4, 1), (257, 33, 5), (4096, 256, 16), (65536, 1024, 64)])
def test_precondition_matches_oracle(rsctx, dtype, tol, n, d, k):
    if dtype == torch.float64 and n * d > 4096 * 256:
        pytest.skip("double GEMM at this size is covered by the float run")
    X = torch.from_numpy(synth.random_matrix(n, d, n + d, scale=1.0 / np.sqrt(d))).to(dtype)
    V = synth.random_orthonormal(d, k, d)
    s2 = synth.random_sigma2(k, k)
    lam = 1e-4
    Vt = torch.from_numpy(V).to(dtype).cuda()
    Z, beta, bh = rs.rs_precondition(rsctx, cuda_rows(X), Vt, torch.from_numpy(s2).cuda(), lam)
    Z = Z.cpu().double().numpy()
    Xd = X.double().numpy()
    Vd = Vt.cpu().double().numpy()
    M = precond.m_matrix(Vd, s2, lam)
    Xt, B = precond.transform(Xd, M)
    Zr, yz, g = precond.components(Xt, B, np.zeros(n), lam)
    scale = np.abs(Xd).max() * (1 + np.sqrt(k))
    np.testing.assert_allclose(Z[:n], Xt, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(Z[n:], B, rtol=0, atol=tol * (1 + np.sqrt(k)))
    beta_ref = precond.smoothness(Zr, g)
    np.testing.assert_allclose(beta.cpu().double().numpy(), beta_ref, rtol=tol * 20 * np.sqrt(d))
    assert bh == pytest.approx(precond.beta_hat(beta_ref), rel=tol * 20 * np.sqrt(d))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("d,k", [(300, 20), (4096, 256), (2050, 129)])
def test_map_output_matches_oracle(rsctx, dtype, tol, d, k):
    """w = M w~ (Eq. (11)); d k <= 65536 takes the one-block kernel, larger maps the many-block one
    (with a ragged last row range at d = 2050)."""
    V = torch.from_numpy(synth.random_orthonormal(d, k, 4)).to(dtype)
    s2 = synth.random_sigma2(k, 2)
    wt = torch.from_numpy(synth.random_vector(d, 3)).to(dtype)
    w = rs.rs_map_output(rsctx, V.cuda(), torch.from_numpy(s2).cuda(), 1e-3, wt.cuda()).cpu().double().numpy()
    ref = precond.m_matrix(V.double().numpy(), s2, 1e-3) @ wt.double().numpy()
    np.testing.assert_allclose(w, ref, rtol=0, atol=tol * 10 * np.abs(ref).max())


@pytest.mark.parametrize("n,d,k", [(3000, 520, 200), (1000, 300, 256), (4100, 1024, 129)])
def test_bf16_components_rank_above_128(rsctx, n, d, k):
    """BF16 data with k in (128, 256]: Z = X - P V^T on tensor cores with two bfloat16 parts of P and V.
    Every entry is within half a bfloat16 ulp of the oracle's M x_i plus the split's dropped terms
    (3 2^-18 |P||V|^T) and the FP32 accumulation (16 u |P||V|^T)."""
    from oracle import precond
    X, _, _ = synth.problem(n, d, np.arange(1, d + 1) ** -1.2, 0.1, n + k)
    Xb = X.to(torch.bfloat16)
    V = synth.random_orthonormal(d, k, k + 1)
    s2 = synth.random_sigma2(k, k + 2)
    lam = 1e-4
    Z, beta, _ = rs.rs_precondition(rsctx, cuda_rows(Xb), torch.from_numpy(V).float().cuda(),
                                    torch.from_numpy(s2).cuda(), lam)
    Vf = torch.from_numpy(V).float().double().numpy()
    M = precond.m_matrix(Vf, s2, lam)
    Xd = Xb.double().numpy()
    ref = Xd @ M
    a = 1.0 - np.sqrt((s2[-1] + lam) / (s2 + lam))
    mag = (np.abs(Xd) @ np.abs(Vf)) * a @ np.abs(Vf).T
    zg = Z[:n].double().cpu().numpy()
    bound = 2.0 ** -8 * np.abs(ref) + (3 * 2.0 ** -18 + 16 * 2.0 ** -24) * mag
    assert np.all(np.abs(zg - ref) <= bound), float(np.max(np.abs(zg - ref) - bound))
