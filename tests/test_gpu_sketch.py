"""GPU parity of the sketch (Alg. 2): range sketch, Cholesky-QR, Jacobi eigensolver, Rayleigh-Ritz
and the composed rs_sketch, against the oracle on the same seeded inputs."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import ridge, sketch as osk
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu


def _data(n, d, alpha, seed, dtype):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -alpha, 0.1, seed)
    return X.to(dtype), y.to(dtype)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 3e-5)])
@pytest.mark.parametrize("kind,n,d,k,s", [("gaussian", 300, 70, 5, 0), ("gaussian", 4096, 256, 16, 0),
                                          ("countsketch", 3000, 130, 12, 256)])
def test_range_sketch_matches_oracle(rsctx, dtype, tol, kind, n, d, k, s):
    X, _ = _data(n, d, 1.5, 11, dtype)
    Y = rs.rs_range_sketch(rsctx, cuda_rows(X), k, 2000, kind=kind, s=s).cpu().double().numpy()
    ref = osk.range_sketch(X.double().numpy(), k, 2000, kind=kind, s=s)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
@pytest.mark.parametrize("d,k", [(10, 1), (70, 9), (1024, 64), (300, 200)])
def test_orthonormalize_matches_oracle(rsctx, dtype, tol, d, k):
    Y = synth.random_matrix(d, k, d + k) @ np.diag(np.logspace(0, -2, k))
    Q = rs.rs_orthonormalize(rsctx, torch.from_numpy(Y).to(dtype).cuda()).cpu().double().numpy()
    Qr = osk.orthonormalize(Y.astype(np.float32).astype(np.float64) if dtype == torch.float32 else Y)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=tol * 10)
    np.testing.assert_allclose(Q, Qr, atol=tol * 100)


def test_orthonormalize_rejects_rank_deficient(rsctx):
    Y = np.ones((20, 3))
    with pytest.raises(rs.RsError):
        rs.rs_orthonormalize(rsctx, torch.from_numpy(Y).cuda())


@pytest.mark.parametrize("prec,tol", [(rs.RS_F64, 1e-12), (rs.RS_F32, 2e-5)])
@pytest.mark.parametrize("k", [1, 2, 7, 16, 64, 97, 128, 256])
def test_sym_eig_matches_library_eigh(rsctx, prec, tol, k):
    G = synth.random_symmetric(k, k, spread=4.0)
    ev, W = rs.rs_sym_eig(rsctx, torch.from_numpy(G).cuda(), prec)
    ev, W = ev.cpu().numpy(), W.cpu().numpy()
    ev_ref, W_ref = osk.sym_eig_desc(G)
    np.testing.assert_allclose(ev, ev_ref, rtol=0, atol=tol * ev_ref[0])
    # invariant checks: W orthonormal and G W = W diag(ev)
    np.testing.assert_allclose(W.T @ W, np.eye(k), atol=tol * 10)
    np.testing.assert_allclose(G @ W, W * ev, atol=tol * 10 * ev_ref[0])


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_ritz_matches_oracle(rsctx, dtype, tol):
    X, _ = _data(2000, 100, 1.2, 3, dtype)
    Q = osk.orthonormalize(synth.random_matrix(100, 10, 1))
    V, s2 = rs.rs_ritz(rsctx, cuda_rows(X), torch.from_numpy(Q).to(dtype).cuda())
    V, s2 = V.cpu().double().numpy(), s2.cpu().numpy()
    Vr, s2r = osk.ritz(X.double().numpy(), Q, 10)
    np.testing.assert_allclose(s2, s2r, rtol=tol)
    np.testing.assert_allclose(V @ np.diag(s2) @ V.T, Vr @ np.diag(s2r) @ Vr.T, atol=tol * s2r[0])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,n,d,k,s,q", [("gaussian", 4096, 256, 16, 0, 1), ("countsketch", 8192, 512, 32, 2048, 1),
                                            ("gaussian", 2048, 128, 8, 0, 3)])
def test_sketch_end_to_end_matches_oracle(rsctx, dtype, kind, n, d, k, s, q):
    """Alg. 2 end to end on the same stored values.  The two sides differ by rounding only: the
    test matrix (float against double Box-Muller draws, about one unit u of the working precision
    per entry), the products forming Y and X Q, and the small eigensolve, each an O(u) relative
    perturbation of the Rayleigh-Ritz matrix, which moves the i-th Ritz value by about
    u sigma_1^2 (absolute) and the preconditioner by about u sigma_1^2 / sigma_k^2 (the
    eigenvector perturbation over the spectral gaps).  CountSketch first sums about n / s rows
    into each bucket, which multiplies the rounding of the sketched data by up to n / s.  Allowed:
    256 u (1 + n / s) sigma_1^2 for the Ritz values and 64 u (1 + n / s) sigma_1^2 / sigma_k^2 for
    M (measured on GB300: at most about a fifth of the first, far below the second)."""
    u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    u = u * (1.0 + n / s) if kind == "countsketch" else u
    X, _ = _data(n, d, 1.5, 21, dtype)
    V, s2 = rs.rs_sketch(rsctx, cuda_rows(X), k, 2000, kind=kind, s=s, q=q)
    V, s2 = V.cpu().double().numpy(), s2.cpu().numpy()
    Vr, s2r = osk.block_lanczos(X.double().numpy(), k, 2000, q=q, kind=kind, s=s)
    # compare the preconditioner M (sign- and rotation-invariant), not V
    from oracle import precond
    M = precond.m_matrix(V, s2, 1e-4)
    Mr = precond.m_matrix(Vr, s2r, 1e-4)
    e_s2, e_m = np.max(np.abs(s2 - s2r)) / s2r[0], np.abs(M - Mr).max()
    print(f"{kind} n={n} d={d} k={k} q={q} {dtype}: max |s2 - s2r| / s2r_0 = {e_s2:.2e}, max |M - Mr| = {e_m:.2e}, "
          f"s2r_0 / s2r_k = {s2r[0] / s2r[-1]:.1f}")
    np.testing.assert_allclose(s2, s2r, rtol=0, atol=256 * u * s2r[0])
    # Ritz values never exceed the true eigenvalues (interlacing)
    lam = np.sort(np.linalg.eigvalsh(ridge.correlation(X.double().numpy())))[::-1]
    assert np.all(s2 <= lam[:k] + 256 * u * lam[0])
    assert e_m <= 64 * u * s2r[0] / s2r[-1], e_m


@pytest.mark.parametrize("n,d,k", [(300, 70, 5), (4096, 256, 16), (5000, 300, 100), (20000, 520, 256), (64, 130, 64)])
def test_tensor_core_range_sketch_bf16_matches_oracle(rsctx, n, d, k):
    """bfloat16 data: Y = X^T Pi on tensor cores with Pi rounded to bfloat16 (the oracle rounds its own
    Philox / Box-Muller values the same way); ragged n, d and k, several 128-column tiles and row
    ranges.  The products are exact in FP32, so only the FP32 accumulation over n rows (and the rare
    entry whose float and double Box-Muller values round to neighbouring bfloat16 values) differ."""
    from oracle import streams
    X, _ = _data(n, d, 1.5, 11, torch.bfloat16)
    Y = rs.rs_range_sketch(rsctx, cuda_rows(X), k, 2000).cpu().double().numpy()
    Xd = X.double().numpy()
    ref = osk.range_sketch(Xd, k, 2000, pi_bf16=True)
    tie, ulp = streams.bf16_rounding_ties(osk.test_matrix_gaussian(2000, n, k))
    allow = np.abs(Xd).T @ (tie * ulp)            # entries that may round the other way
    assert np.all(np.abs(Y - ref) <= 3e-5 * np.abs(ref).max() + allow), np.max(np.abs(Y - ref) - allow)


def test_tensor_core_range_sketch_can_be_switched_off(rsctx, monkeypatch):
    """RS_UMMA_SKETCH=0 selects the CUDA-core sketch with the float test matrix (the oracle's Pi)."""
    monkeypatch.setenv("RS_UMMA_SKETCH", "0")
    X, _ = _data(3000, 200, 1.5, 12, torch.bfloat16)
    Y = rs.rs_range_sketch(rsctx, cuda_rows(X), 24, 2000).cpu().double().numpy()
    ref = osk.range_sketch(X.double().numpy(), 24, 2000)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=3e-5 * np.abs(ref).max())


@pytest.mark.parametrize("k,spread", [(64, 5.0), (256, 5.0), (200, 8.0)])
def test_sym_eig_float_keeps_relative_accuracy_of_small_eigenvalues(rsctx, k, spread):
    """Graded spectra (eigenvalues over 10^spread) in a random basis: the float eigen-solve returns
    every eigenvalue, the smallest included, to a relative 1e-4 (a float Jacobi with an absolute
    floor alone would leave the small ones with absolute accuracy only)."""
    G = synth.random_symmetric(k, k + 7, spread=spread)
    ev, W = rs.rs_sym_eig(rsctx, torch.from_numpy(G).cuda(), rs.RS_F32)
    ev_ref, _ = osk.sym_eig_desc(G)
    np.testing.assert_allclose(ev.cpu().numpy(), ev_ref, rtol=1e-4)
