"""The allocation-free full-gradient entry point (rs_full_gradient_static) against the regular one.

Callers that own all device memory through their own pool, or that must stay off the driver's
allocation path, use rs_full_gradient_static: it takes no context and keeps its partial sums in
a fixed array in the library's device data.  This file is collected last on purpose, so that a
run stopping at the first failure has already run every other test; it also passes alone.
"""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import precond
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


def _components(n, d, seed, dtype, lam):
    Z = synth.random_matrix(n + d, d, seed, scale=1.0 / np.sqrt(d))
    Zt = torch.from_numpy(Z).to(dtype)
    ld = ((d * Zt.element_size() + 15) // 16 * 16) // Zt.element_size()
    buf = torch.zeros(n + d, ld, dtype=dtype)
    buf[:, :d] = Zt
    y = torch.from_numpy(synth.random_vector(n, seed + 1)).to(dtype)
    return buf.cuda()[:, :d], y.cuda()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("n,d", [(5000, 37), (65536, 1024)])
def test_static_entry_matches_regular_entry_twice(rsctx, dtype, tol, n, d):
    if dtype == torch.float64 and d > 512:
        d = 512
    lam = 1e-3
    Z, y = _components(n, d, n + d, dtype, lam)
    w = torch.from_numpy(synth.random_vector(d, 1)).to(dtype).cuda()
    ref = rs.rs_full_gradient(rsctx, Z, y, n, lam, w)
    scale = float(ref.abs().max())
    out = torch.empty_like(ref)
    for _ in range(2):      # the shared array keeps the previous call's contents
        out.fill_(float("nan"))
        got = rs.rs_full_gradient_static(Z, y, n, lam, w, stream=rsctx.stream, out=out)
        torch.cuda.synchronize()
        err = float((got - ref).abs().max())
        assert err <= tol * max(scale, 1e-30), err
    # the oracle agrees too (same scale as the regular parity test)
    Zd = Z.double().cpu().numpy()
    _, yz, g = precond.components(Zd[:n], Zd[n:], y.double().cpu().numpy(), lam)
    from oracle import svrg
    mu_ref = svrg.full_gradient_fast(Zd, yz, g, w.double().cpu().numpy())
    assert np.abs(got.double().cpu().numpy() - mu_ref).max() <= 100 * tol * max(np.abs(mu_ref).max(), 1e-30)


def test_static_entry_rejects_rows_beyond_its_limit(rsctx):
    n, d = 100, 1028
    Z, y = _components(n, d, 3, torch.float32, 1e-3)
    w = torch.zeros(d, device="cuda")
    with pytest.raises(rs.RsError) as e:
        rs.rs_full_gradient_static(Z, y, n, 1e-3, w, out=torch.empty(d, device="cuda"))
    assert e.value.code == 1 and "maximum" in str(e.value)


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float8_e4m3fn])
def test_static_entry_refuses_narrow_rows_before_launching(rsctx, dtype):
    """BF16 / FP8 rows have no kernel in the allocation-free entry: the call must return RS_EINVAL
    from its host-side checks and leave mu untouched (no kernel ran)."""
    n, d = 256, 64
    Z = torch.zeros(n + d, d, dtype=dtype, device="cuda")
    y = torch.zeros(n, device="cuda")
    w = torch.zeros(d, device="cuda")
    mu = torch.full((d,), float("nan"), device="cuda")
    with pytest.raises(rs.RsError) as e:
        rs.rs_full_gradient_static(Z, y, n, 1e-3, w, out=mu)
    assert e.value.code == 1
    if dtype == torch.bfloat16:
        assert "RS_F32" in str(e.value)
    torch.cuda.synchronize()
    assert torch.isnan(mu).all()
