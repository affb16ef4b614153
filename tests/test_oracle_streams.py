"""Pins for oracle.streams: Philox4x32-10 against an independent library implementation,
distributional checks of every draw, exact integer arithmetic of the sampler."""

from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import streams


def _triton_philox(counters, seed):
    """Philox4x32-10 words from triton's implementation, run by its CPU interpreter."""
    tp = pytest.importorskip("tests._triton_philox")
    return tp.philox_words(counters, seed)


def test_philox_matches_triton_reference_implementation():
    rng = np.random.default_rng(1)
    counters = rng.integers(0, 2 ** 32, (64, 4), dtype=np.uint64)
    counters[0] = 0
    counters[1] = 2 ** 32 - 1
    for seed in (0, 12345, 2 ** 64 - 1, 0x0123456789ABCDEF):
        ref = _triton_philox(counters, seed)
        got = np.stack(streams.philox4x32_10(*counters.T, seed), axis=1)
        np.testing.assert_array_equal(got, ref)


def test_philox_bits_are_balanced_and_distinct():
    i = np.arange(1 << 16, dtype=np.uint64)
    w = np.stack(streams.philox4x32_10(i, 0, 7, 3, 99), axis=1)
    bits = np.unpackbits(w.view(np.uint8))
    # 2^21 bits: mean within 5 sigma of 1/2
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / np.sqrt(bits.size)
    # a bijection of the counter for a fixed key: no repeated 128-bit outputs
    assert len({tuple(r) for r in w}) == w.shape[0]
    # neighbouring keys and counters decorrelate
    w2 = np.stack(streams.philox4x32_10(i, 0, 7, 3, 100), axis=1)
    assert np.mean(w == w2) < 1e-3


def test_uniform24_range_and_float32_exact():
    w = np.array([0, 511, 512, 2 ** 32 - 1], dtype=np.uint32)
    u = streams.uniform24(w)
    assert u[0] == 2.0 ** -24 and u[1] == u[0]
    assert u[2] == 3.0 * 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    uu = streams.uniform24(np.random.default_rng(0).integers(0, 2 ** 32, 100000, dtype=np.uint64).astype(np.uint32))
    assert np.all(uu.astype(np.float32).astype(np.float64) == uu)
    assert stats.kstest(uu, "uniform").pvalue > 1e-4


def test_box_muller_special_values_and_distribution():
    z0, z1 = streams.box_muller(np.array([np.exp(-0.5)]), np.array([0.0]))
    assert z0[0] == pytest.approx(1.0, abs=1e-15) and z1[0] == pytest.approx(0.0, abs=1e-15)
    z0, z1 = streams.box_muller(np.array([np.exp(-2.0)]), np.array([0.25]))
    assert z0[0] == pytest.approx(0.0, abs=1e-15) and z1[0] == pytest.approx(2.0, abs=1e-15)
    G = streams.gaussian(2024, 4096, 50)
    assert G.shape == (4096, 50)
    x = G.ravel()
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # columns are uncorrelated
    c = np.corrcoef(G[:, :8].T)
    assert np.max(np.abs(c - np.eye(8))) < 6 / np.sqrt(4096)


def test_gaussian_is_counter_addressed():
    full = streams.gaussian(7, 100, 10)
    part = streams.gaussian(7, 30, 10, row0=50)
    np.testing.assert_array_equal(full[50:80], part)
    np.testing.assert_array_equal(streams.gaussian(7, 100, 6), full[:, :6])


def test_countsketch_hash_range_and_balance():
    b, s = streams.countsketch_hash(11, 100000, 64)
    assert b.min() >= 0 and b.max() < 64
    assert set(np.unique(s)) == {-1.0, 1.0}
    counts = np.bincount(b, minlength=64)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert abs(s.mean()) < 5 / np.sqrt(s.size)


def test_quantize_weights_exact_values():
    beta = np.array([4.0, 2.0, 1.0, 0.0, 4.0 * 2.0 ** -24, 4.0 * 2.0 ** -30])
    W = streams.quantize_weights(beta)
    np.testing.assert_array_equal(W, [1 << 24, 1 << 23, 1 << 22, 1, 1, 1])
    with pytest.raises(ValueError):
        streams.quantize_weights([1.0, np.nan])


def test_sampler_semantics_against_brute_force():
    W = np.array([3, 1, 0 + 1, 5, 2], dtype=np.uint32)
    cum = streams.cumulative(W)
    assert cum.tolist() == [3, 4, 5, 10, 12]
    T = int(cum[-1])
    t = np.arange(200, dtype=np.uint64)
    w0, w1, _, _ = streams.philox4x32_10(t, 0, 4, streams.TAG_SAMPLE, 77)
    idx = streams.sample_indices(cum, 77, 4, 200)
    for k in range(200):
        u = (int(w1[k]) << 32) | int(w0[k])
        r = Fraction(u * T, 2 ** 64)
        r = r.numerator // r.denominator
        # brute force: the first i whose cumulative weight exceeds r
        i = next(j for j in range(len(W)) if int(cum[j]) > r)
        assert idx[k] == i


def test_sampler_frequencies_follow_q():
    W = np.array([1, 2, 4, 8, 16, 32, 64, 128], dtype=np.uint32)
    cum = streams.cumulative(W)
    idx = streams.sample_indices(cum, 5, 0, 60000)
    counts = np.bincount(idx, minlength=8)
    assert stats.chisquare(counts, 60000 * W / W.sum()).pvalue > 1e-4
    iu = streams.sample_indices_uniform(10, 5, 1, 50000)
    assert iu.min() >= 0 and iu.max() < 10
    assert stats.chisquare(np.bincount(iu, minlength=10)).pvalue > 1e-4


def test_gaussian_column_subset_equals_the_full_matrix_columns():
    from oracle import streams as st
    full = st.gaussian(99, 37, 11, row0=5)
    cols = [10, 0, 3, 4, 7]
    np.testing.assert_array_equal(st.gaussian_columns(99, 37, cols, row0=5), full[:, cols])


def test_round_bf16_matches_the_bit_level_rounding():
    """Nearest-even rounding to 8 significant bits, checked against the float32 bit manipulation
    (add 0x7FFF plus the lowest kept bit, clear the low 16 bits) on float32 inputs, ties included."""
    from oracle import streams as st
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(20000), rng.standard_normal(20000) * 1e3]).astype(np.float32)
    m = np.arange(0, 128, dtype=np.uint32)
    ties = ((np.uint32(127 + 3) << 23) | (m << 16) | 0x8000).view(np.float32)      # exact halfway points
    x = np.concatenate([x, ties, -ties])
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    ref = b.astype(np.uint32).view(np.float32).astype(np.float64)
    np.testing.assert_array_equal(st.round_bf16(x.astype(np.float64)), ref)


def test_bf16_rounding_ties_flags_exactly_the_near_midpoint_entries():
    from oracle import streams as st
    ulp = 2.0 ** -7                                   # bfloat16 spacing in [1, 2)
    mid = 1.0 + 37.5 * ulp                            # a rounding midpoint
    x = np.array([mid, mid * (1 + 2 ** -22), mid * (1 + 2 ** -18), 1.0 + 37 * ulp, -mid])
    tie, step = st.bf16_rounding_ties(x)
    assert tie.tolist() == [True, True, False, False, True]
    np.testing.assert_array_equal(step, np.full(5, ulp))
    # values a margin away from the midpoint round to the same neighbour on both sides of the margin
    lo, hi = mid * (1 - 2 ** -21), mid * (1 + 2 ** -21)
    assert st.round_bf16(np.array([lo]))[0] != st.round_bf16(np.array([hi]))[0]
