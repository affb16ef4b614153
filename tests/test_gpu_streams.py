"""GPU parity of the random streams (Philox words, Gaussian test matrix, CountSketch hash and sums,
integer sampling weights, prefix table, index stream) against the oracle, through the C ABI."""

import numpy as np
import pytest
import torch

import paper_1602_02350_gb300 as rs
from oracle import sketch as osk
from oracle import streams
from paper_1602_02350_gb300 import synth

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed,c2,c3,count", [(0, 0, 0, 1), (12345, 7, 3, 1000), (2 ** 64 - 1, 2 ** 32 - 1, 1, 4099)])
def test_philox_words_bit_exact(rsctx, seed, c2, c3, count):
    got = _u32(rs.rs_philox_words(rsctx, seed, c2, c3, count)).reshape(count, 4)
    i = np.arange(count, dtype=np.uint64)
    ref = np.stack(streams.philox4x32_10(i & np.uint64(0xFFFFFFFF), i >> np.uint64(32), c2, c3, seed), axis=1)
    np.testing.assert_array_equal(got, ref)


def _ulp32(x):
    return np.spacing(np.abs(x).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("rows,cols,row0", [(1, 1, 0), (257, 13, 5), (4096, 64, 1 << 33)])
def test_gaussian_matches_oracle(rsctx, rows, cols, row0):
    ref = streams.gaussian(2001, rows, cols, row0=row0)
    g64 = rs.rs_gaussian(rsctx, 2001, rows, cols, torch.float64, row0=row0).cpu().numpy()
    np.testing.assert_allclose(g64, ref, rtol=1e-14, atol=1e-14)
    g32 = rs.rs_gaussian(rsctx, 2001, rows, cols, torch.float32, row0=row0).cpu().numpy().astype(np.float64)
    # float transcendentals: within 4 float ulps of the double value
    assert np.all(np.abs(g32 - ref) <= 4 * _ulp32(ref) + 1e-30)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,d,s", [(1, 4, 1), (1000, 36, 64), (65536, 1024, 4096)])
def test_countsketch_hash_bit_exact_and_sums(rsctx, dtype, n, d, s):
    X = torch.from_numpy(synth.random_matrix(n, d, 5)).to(dtype)
    SX, bucket, sign = rs.rs_countsketch(rsctx, X.cuda(), 77, s, with_hash=True)
    b_ref, s_ref = streams.countsketch_hash(77, n, s)
    np.testing.assert_array_equal(bucket.cpu().numpy(), b_ref)
    np.testing.assert_array_equal(sign.cpu().numpy(), s_ref)
    if n * d <= 40000:
        ref = osk.countsketch_rows(X.double().numpy(), 77, s)
    else:  # the same sums as a sparse-times-dense product (library routine)
        from scipy import sparse
        S = sparse.csr_matrix((s_ref, (b_ref, np.arange(n))), shape=(s, n))
        ref = S @ X.double().numpy()
    # recursive summation of c terms: |error| <= c u sum|terms| <= c^2 u max|x|
    u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    c = np.bincount(b_ref, minlength=s).max()
    np.testing.assert_allclose(SX.cpu().double().numpy(), ref, rtol=0,
                               atol=u * c * c * np.abs(X.double().numpy()).max())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("N", [1, 5, 1025, 66560])
def test_sampling_weights_and_table_bit_exact(rsctx, dtype, N):
    beta = torch.from_numpy(np.abs(synth.random_vector(N, N)) ** 3).to(dtype)
    if N > 3:
        beta[2] = 0.0
    W = rs.rs_sampling_weights(rsctx, beta.cuda())
    W_ref = streams.quantize_weights(beta.double().numpy())
    np.testing.assert_array_equal(_u32(W), W_ref)
    cum = rs.rs_sampling_table(rsctx, W).cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(cum, streams.cumulative(W_ref))


def test_sampling_weights_reject_nonfinite(rsctx):
    beta = torch.tensor([1.0, float("nan"), 2.0], dtype=torch.float32, device="cuda")
    with pytest.raises(rs.RsError) as e:
        rs.rs_sampling_weights(rsctx, beta)
    assert e.value.code == 4


@pytest.mark.parametrize("N,m,epoch,t0", [(1, 3, 0, 0), (7, 1000, 2, 0), (66560, 131072, 5, 0), (4352, 300, 9, 8192)])
def test_index_stream_bit_exact(rsctx, N, m, epoch, t0):
    W_ref = synth.random_weights(N, 3 + N)
    cum_ref = streams.cumulative(W_ref)
    W = torch.from_numpy(W_ref.view(np.int32)).cuda()
    cum = torch.from_numpy(cum_ref.view(np.int64)).cuda()
    idx, inq = rs.rs_index_stream(rsctx, W, cum, N, 3001, epoch, m, t0=t0, dtype=torch.float64)
    ref = streams.sample_indices(cum_ref, 3001, epoch, m, t0=t0)
    np.testing.assert_array_equal(_u32(idx).astype(np.int64), ref)
    T = float(cum_ref[-1])
    np.testing.assert_allclose(inq.cpu().numpy(), T / (N * W_ref[ref].astype(np.float64)), rtol=1e-15)
    idx32, inq32 = rs.rs_index_stream(rsctx, W, cum, N, 3001, epoch, m, t0=t0, dtype=torch.float32)
    np.testing.assert_array_equal(_u32(idx32).astype(np.int64), ref)
    np.testing.assert_allclose(inq32.cpu().numpy(), T / (N * W_ref[ref].astype(np.float64)), rtol=1e-7)


def test_uniform_index_stream_bit_exact(rsctx):
    idx, inq = rs.rs_index_stream(rsctx, None, None, 1000, 5, 1, 5000, sampling=rs.RS_SAMPLE_UNIFORM)
    np.testing.assert_array_equal(_u32(idx).astype(np.int64), streams.sample_indices_uniform(1000, 5, 1, 5000))
    assert torch.all(inq == 1)
