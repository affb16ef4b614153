"""GPU parity of the speed-up diagnostic (the ratio after Thm 1, Fig. 1) against the oracle: the
kernel on given sketched eigenvalues, and end to end from a sketch of data through the C ABI."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import ridge, sketch as osk
from paper_1602_02350_gb300 import synth
from tests.gpu_helpers import cuda_rows

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K", [1, 7, 64, 256, 4096])
def test_ratio_kernel_matches_oracle(rsctx, K):
    s2 = synth.random_sigma2(K, K, lo=1e-6, hi=10.0)
    trc = float(s2.sum() * 1.7)          # a tail beyond the K sketched values
    r, ra = rs.rs_speedup_ratio(rsctx, torch.from_numpy(s2).cuda(), trc)
    r, ra = r.cpu().numpy(), ra.cpu().numpy()
    ref = np.array([ridge.speedup_ratio_sketched(s2, trc, k) for k in range(1, K + 1)])
    np.testing.assert_allclose(r, ref, rtol=1e-13)
    np.testing.assert_allclose(ra, np.sqrt(ref), rtol=1e-13)


def test_ratio_rejects_bad_arguments(rsctx):
    s2 = torch.ones(4, dtype=torch.float64, device="cuda")
    for trc in (0.0, -1.0, float("nan")):
        with pytest.raises(rs.RsError) as e:
            rs.rs_speedup_ratio(rsctx, s2, trc)
        assert e.value.code == 1


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 2e-4)])
def test_ratio_from_sketch_matches_oracle(rsctx, dtype, tol):
    """rs_sketch (rank 64) + rs_trace_c + rs_speedup_ratio on the device against the oracle's own
    sketch and tr(C) of the same data; with fast decay (alpha = 2) the ratio is large for small k."""
    n, d, K = 8192, 512, 64
    X, _, _ = synth.problem(n, d, np.arange(1, d + 1) ** -2.0, 0.1, 31)
    Xt = X.to(dtype)
    Xc = cuda_rows(Xt)
    _, s2 = rs.rs_sketch(rsctx, Xc, K, 2000)
    trc = rs.rs_trace_c(rsctx, Xc)
    r, _ = rs.rs_speedup_ratio(rsctx, s2, trc)
    Xd = Xt.double().numpy()
    _, s2r = osk.block_lanczos(Xd, K, 2000)
    trr = float((Xd * Xd).sum() / n)
    assert trc == pytest.approx(trr, rel=1e-12 if dtype == torch.float64 else 1e-6)
    ref = np.array([ridge.speedup_ratio_sketched(s2r, trr, k) for k in range(1, K + 1)])
    # ratio(k) = T / den with den = k s_k + T - S_k: relative errors eps_r in the Ritz values move den
    # by at most eps_r (S_k + k s_k) <= 2 eps_r T, i.e. ratio(k) by a relative 2 eps_r ratio(k);
    # eps_r ~ 4 K u for float data (Cholesky-QR's float factorisation), the tolerance for double
    eps_r = tol if dtype == torch.float64 else 4 * K * 2.0 ** -24
    got = r.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2 * eps_r * ref * ref + 1e-12), np.max(np.abs(got - ref) / (ref * ref))
    assert ref[31] > 5.0 * ref[0]


def test_bounded_wait_gives_up_and_the_context_survives(rsctx):
    """A device-side wait that nothing completes gives up after its budget (about 2 ms here), the call
    reports RS_ETIMEOUT (5), and the same context then runs ordinary work correctly."""
    rs.rs_wait_probe(rsctx, 4_000_000, True)
    with pytest.raises(rs.RsError) as e:
        rs.rs_wait_probe(rsctx, 4_000_000, False)
    assert e.value.code == 5 and "gave up" in str(e.value)
    s2 = torch.tensor([4.0, 1.0], dtype=torch.float64, device="cuda")
    r, _ = rs.rs_speedup_ratio(rsctx, s2, 6.0)
    np.testing.assert_allclose(r.cpu().numpy(), [1.0, 6.0 / (2.0 + 1.0)], rtol=1e-15)
    with pytest.raises(rs.RsError) as e:
        rs.rs_wait_probe(rsctx, 0, True)
    assert e.value.code == 1
