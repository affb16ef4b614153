"""CPU checks of numerical devices the CUDA kernels rely on (float64 / exact emulation, no GPU):
the three-part bfloat16 split of float operands and the six retained products of the tensor-core
contractions, the round-robin pairing of the Jacobi eigensolver, and the shuffle reduce-scatter
of the skinny X U pass."""

import itertools

import numpy as np
import pytest


def _bf16(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float32 (finite inputs)."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split3(x):
    """x = x0 + x1 + x2 with x_p = bf16(x - x0 - .. - x_{p-1}), residuals in float32 (as the kernels)."""
    x = np.asarray(x, np.float32)
    x0 = _bf16(x)
    r = (x - x0).astype(np.float32)
    x1 = _bf16(r)
    r = (r - x1).astype(np.float32)
    x2 = _bf16(r)
    return x0, x1, x2


@pytest.mark.parametrize("scale", [1e-20, 1e-3, 1.0, 1e4, 1e30])
def test_three_part_split_reproduces_float(scale):
    """(While the third part stays a normal float, |x| above about 2^-110.)"""
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100000) * scale).astype(np.float32)
    x0, x1, x2 = _split3(x)
    err = np.abs(x.astype(np.float64) - (x0.astype(np.float64) + x1 + x2))
    # 24 significant bits in three parts of 8: the remainder is below half an ulp of the third part
    assert np.all(err <= 2.0 ** -24 * np.abs(x.astype(np.float64)))
    # the first two parts add exactly in float32 (at most 16 significant bits)
    assert np.array_equal((x0 + x1).astype(np.float64), x0.astype(np.float64) + x1.astype(np.float64))


def test_six_products_keep_float_accuracy():
    """sum over a + b <= 2 of P_a V_b^T (the products the components and X W kernels issue) is
    within a few 2^-24 of P V^T relative to |P| |V|^T; dropping the a + b = 2 terms is not."""
    rng = np.random.default_rng(5)
    n, d, k = 200, 150, 64
    P = rng.standard_normal((n, k)).astype(np.float32)
    V = (rng.standard_normal((d, k)) / np.sqrt(k)).astype(np.float32)
    Pp = [p.astype(np.float64) for p in _split3(P)]
    Vp = [v.astype(np.float64) for v in _split3(V)]
    exact = P.astype(np.float64) @ V.astype(np.float64).T
    mag = np.abs(P.astype(np.float64)) @ np.abs(V.astype(np.float64)).T
    six = sum(Pp[a] @ Vp[b].T for a in range(3) for b in range(3) if a + b <= 2)
    three = sum(Pp[a] @ Vp[b].T for a in range(2) for b in range(2) if a + b <= 1)
    assert np.max(np.abs(six - exact) / mag) <= 4 * 2.0 ** -24
    assert np.max(np.abs(three - exact) / mag) > 16 * 2.0 ** -24


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16, 63, 64, 97, 128])
def test_jacobi_round_robin_pairs_every_plane_once_per_sweep(k):
    """Seats pos(j) = ((j - 1 + r) mod (K - 1)) + 1, computed by one conditional subtraction, pair
    players i and K - 1 - i; over the K - 1 rounds each pair {p, q} of the K players meets once."""
    K = (k + 1) & ~1
    seen = []
    for r in range(K - 1):
        def pos(j):
            if j == 0:
                return 0
            v = j - 1 + r
            assert v < 2 * (K - 1)
            return (v - (K - 1) if v >= K - 1 else v) + 1
        rnd = [tuple(sorted((pos(i), pos(K - 1 - i)))) for i in range(K // 2)]
        assert sorted(x for pr in rnd for x in pr) == list(range(K))   # disjoint planes in a round
        seen += rnd
    assert sorted(seen) == sorted(itertools.combinations(range(K), 2))


def test_shuffle_reduce_scatter_leaves_value_index_lane_on_lane():
    """Five butterfly steps with halving payloads: lane L ends with the sum over lanes of value L."""
    rng = np.random.default_rng(9)
    vals = rng.standard_normal((32, 32))            # vals[lane][index]
    v = [list(row) for row in vals]
    for s in range(5):
        o = 16 >> s
        send = [[(v[L][k] if (L & o) else v[L][k + o]) for k in range(o)] for L in range(32)]
        keep = [[(v[L][k + o] if (L & o) else v[L][k]) for k in range(o)] for L in range(32)]
        v = [[keep[L][k] + send[L ^ o][k] for k in range(o)] for L in range(32)]
    got = np.array([v[L][0] for L in range(32)])
    np.testing.assert_allclose(got, vals.sum(axis=0), rtol=1e-12)
