"""Counter-based random streams, float64 / exact integers (oracle; test infrastructure).

The method draws three kinds of random numbers: the Gaussian test matrix of
Alg. 2, the CountSketch hash that can precede it, and the index i_t that Alg. 1
samples with probability q_i each inner step.  Both the oracle and the CUDA path
derive them from one counter-based generator, Philox4x32-10 (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), so the two
sides agree on every draw without sharing code.  This file is written from the
published definition of that generator.

Stream layout (counter words c0..c3, key = the 64-bit seed split lo/hi):

  Gaussian entry (i, 4g + r):   c = (lo32(i), hi32(i), g, TAG_GAUSS),     r = 0..3
  CountSketch hash of row i:    c = (lo32(i), hi32(i), 0, TAG_COUNTSKETCH)
  sampled index of step t in
  epoch e:                      c = (lo32(t), hi32(t), e, TAG_SAMPLE)
"""

import numpy as np

TAG_GAUSS = 1
TAG_COUNTSKETCH = 2
TAG_SAMPLE = 3

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)   # Philox-4x32 round multipliers
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)   # Weyl key increments (golden ratio, sqrt(3) - 1)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, seed):
    """Philox4x32 with 10 rounds on counter arrays (c0, c1, c2, c3) and a 64-bit key.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
        (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
    and the key is advanced by the Weyl constants between rounds.
    Returns four uint32 arrays.
    """
    shape = np.broadcast(np.asarray(c0), np.asarray(c1), np.asarray(c2), np.asarray(c3)).shape
    x0, x1, x2, x3 = (np.broadcast_to(np.asarray(c, dtype=np.uint64) & _MASK, shape).copy()
                      for c in (c0, c1, c2, c3))
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64(seed >> 32)
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        x0, x1, x2, x3 = ((p1 >> np.uint64(32)) ^ x1 ^ k0, p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ x3 ^ k1, p0 & _MASK)
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return tuple(x.astype(np.uint32) for x in (x0, x1, x2, x3))


def uniform24(w):
    """Map a uint32 word to (2m + 1) 2^-24 with m its top 23 bits: a uniform on (0, 1)
    that is exactly representable in float32 (24-bit significand) and never 0 or 1."""
    m = (np.asarray(w, np.uint32) >> np.uint32(9)).astype(np.float64)
    return (2.0 * m + 1.0) * 2.0 ** -24


def box_muller(ua, ub):
    """Two independent N(0,1) draws from two uniforms (Box and Muller, 1958)."""
    rho = np.sqrt(-2.0 * np.log(ua))
    return rho * np.cos(2.0 * np.pi * ub), rho * np.sin(2.0 * np.pi * ub)


def gaussian(seed, rows, cols, row0=0):
    """Gaussian matrix G[i, j], i in [row0, row0 + rows), j < cols; N(0,1) entries.

    Entry (i, 4g + r) comes from the words of counter (i, g, TAG_GAUSS):
    words (0,1) -> entries r = 0,1 and words (2,3) -> r = 2,3 by Box-Muller.
    """
    groups = (cols + 3) // 4
    i = np.arange(row0, row0 + rows, dtype=np.uint64)[:, None]
    g = np.arange(groups, dtype=np.uint64)[None, :]
    w0, w1, w2, w3 = philox4x32_10(i & _MASK, i >> np.uint64(32), g, TAG_GAUSS, seed)
    z0, z1 = box_muller(uniform24(w0), uniform24(w1))
    z2, z3 = box_muller(uniform24(w2), uniform24(w3))
    out = np.stack([z0, z1, z2, z3], axis=-1).reshape(rows, groups * 4)
    return out[:, :cols].copy()


def round_bf16(x):
    """Nearest bfloat16 value (8 significant bits, ties to even) of each float64 entry, as float64:
    x = m 2^e with m in [0.5, 1), rounded to m' = rint(256 m) / 256 (normal range)."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def bf16_rounding_ties(x, margin=2.0 ** -20):
    """(mask, ulp): entries whose float64 value lies within ``margin`` |x| of a bfloat16 rounding
    midpoint, where a float computation of the same value (a few float ulps away) may round to the
    neighbouring bfloat16 value, and the bfloat16 spacing at x (the size of that disagreement)."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    frac = np.abs(m) * 256.0
    dist = np.abs(frac - np.floor(frac) - 0.5)          # distance to the midpoint, in ulps
    ulp = np.ldexp(1.0, e - 8)
    return dist * ulp <= margin * np.abs(x), ulp


def gaussian_columns(seed, rows, cols, row0=0, bf16=False):
    """Columns ``cols`` (any subset, any order) of the same Gaussian matrix as ``gaussian`` (entries
    rounded by ``round_bf16`` when ``bf16``):
    column j = 4g + r is entry r of the Box-Muller pairs of counter (i, g, TAG_GAUSS), so only the
    counters of the groups g the columns fall in are evaluated."""
    cols = np.asarray(cols, np.int64)
    out = np.empty((rows, cols.size))
    i = np.arange(row0, row0 + rows, dtype=np.uint64)
    for c, j in enumerate(cols):
        g = np.uint64(j // 4)
        w0, w1, w2, w3 = philox4x32_10(i & _MASK, i >> np.uint64(32), g, TAG_GAUSS, seed)
        r = int(j % 4)
        if r < 2:
            z = box_muller(uniform24(w0), uniform24(w1))
        else:
            z = box_muller(uniform24(w2), uniform24(w3))
        out[:, c] = z[r % 2]
    return round_bf16(out) if bf16 else out


def countsketch_hash(seed, n, s):
    """Bucket h(i) in [0, s) and sign sigma(i) in {+1, -1} for rows i < n.

    h(i) = floor(w0 * s / 2^32) (exact integer product), sigma(i) = -1 iff the top bit of w1 is set.
    """
    i = np.arange(n, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(i & _MASK, i >> np.uint64(32), 0, TAG_COUNTSKETCH, seed)
    bucket = ((w0.astype(np.uint64) * np.uint64(s)) >> np.uint64(32)).astype(np.int64)
    sign = np.where((w1 >> np.uint32(31)) != 0, -1.0, 1.0)
    return bucket, sign


def quantize_weights(beta):
    """Integer sampling weights W_i = max(1, floor(2^24 beta_i / max_j beta_j)).

    The division is one correctly rounded float64 operation and the scaling by
    2^24 is exact, so any implementation given the same beta values gets the
    same integers.  q_i = W_i / sum_j W_j is then an exact rational that both
    sides share (the reading of "q_i = beta_i / sum beta_j" in Alg. 1 and
    Alg. 3 that makes the index stream reproducible bit for bit).
    """
    b = np.asarray(beta, np.float64)
    if not np.all(np.isfinite(b)) or np.any(b < 0):
        raise ValueError("smoothness constants must be finite and non-negative")
    bmax = b.max()
    if bmax <= 0:
        return np.ones(b.shape, np.uint32)
    W = np.floor(np.ldexp(b / bmax, 24))
    return np.maximum(W, 1.0).astype(np.uint32)


def cumulative(W):
    """Inclusive prefix sums cum[i] = W_0 + ... + W_i as exact uint64."""
    return np.cumsum(np.asarray(W, np.uint64), dtype=np.uint64)


def sample_indices(cum, seed, epoch, m, t0=0):
    """Indices i_t, t in [t0, t0 + m), drawn with probability q_i = W_i / T (Alg. 1).

    u = w1 2^32 + w0 is a uniform 64-bit integer; r = floor(u T / 2^64) is then
    uniform on [0, T) up to a bias below T / 2^64; i_t is the smallest i with
    cum[i] > r.  The product is formed exactly with Python integers.
    """
    cum = np.asarray(cum, np.uint64)
    T = int(cum[-1])
    t = np.arange(t0, t0 + m, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(t & _MASK, t >> np.uint64(32), int(epoch), TAG_SAMPLE, seed)
    u = (w1.astype(object) << 32) | w0.astype(object)
    r = np.array([(int(v) * T) >> 64 for v in u], dtype=np.uint64)
    return np.searchsorted(cum, r, side="right").astype(np.int64)


def sample_indices_uniform(N, seed, epoch, m, t0=0):
    """Uniform sampling (the original SVRG of Johnson and Zhang, Sec. 4.2): i_t = floor(w0 N / 2^32)."""
    t = np.arange(t0, t0 + m, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(t & _MASK, t >> np.uint64(32), int(epoch), TAG_SAMPLE, seed)
    return ((w0.astype(np.uint64) * np.uint64(N)) >> np.uint64(32)).astype(np.int64)
