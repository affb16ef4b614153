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


def _packed_jacobi(G, tol=1e-6, floor_ulps=8.0, max_sweeps=30):
    """float32 emulation of the packed one-pass Jacobi rounds (rotation choice, then every 2 x 2 block
    of the round's disjoint planes rotated from both sides; diagonal blocks by the closed form), with
    the rotation log replayed onto the identity afterwards, as the kernels do."""
    k = G.shape[0]
    K = (k + 1) & ~1
    P = K // 2
    A = G.astype(np.float32).copy()
    u = np.float32(2.0 ** -24)
    floor = np.float32(floor_ulps * np.linalg.norm(G) * 2.0 ** -24)
    log = []
    for _ in range(max_sweeps):
        rotated = False
        for r in range(K - 1):
            def pos(j):
                if j == 0:
                    return 0
                v = j - 1 + r
                return (v - (K - 1) if v >= K - 1 else v) + 1
            pairs = []
            for i in range(P):
                p, q = sorted((pos(i), pos(K - 1 - i)))
                c, s, t = np.float32(1), np.float32(0), np.float32(0)
                if q < k:
                    app, aqq, apq = A[p, p], A[q, q], A[q, p]
                    noise = np.float32(4) * u * max(abs(app), abs(aqq))
                    thr = max(np.float32(tol) * np.sqrt(abs(app * aqq)), floor, noise)
                    if abs(apq) > thr:
                        theta = (aqq - app) / (np.float32(2) * apq)
                        t = np.float32((1 if theta >= 0 else -1) / (abs(theta) + np.sqrt(theta * theta + 1)))
                        c = np.float32(1 / np.sqrt(t * t + 1))
                        s = np.float32(t * c)
                        rotated = True
                pairs.append((p, q, c, s, t))
            log.append(pairs)
            Anew = A.copy()
            for a in range(P):
                for b in range(a + 1):
                    pa, qa, ca, sa, ta = pairs[a]
                    pb, qb, cb, sb, tb = pairs[b]
                    if sa == 0 and sb == 0:
                        continue
                    if a == b:
                        apq = A[qa, pa]
                        Anew[pa, pa] = A[pa, pa] - ta * apq
                        Anew[qa, qa] = A[qa, qa] + ta * apq
                        Anew[qa, pa] = Anew[pa, qa] = 0
                        continue
                    ra, rb = qa < k, qb < k
                    m = np.zeros((2, 2), np.float32)
                    m[0, 0] = A[pa, pb]
                    m[0, 1] = A[pa, qb] if rb else 0
                    m[1, 0] = A[qa, pb] if ra else 0
                    m[1, 1] = A[qa, qb] if ra and rb else 0
                    Ra = np.array([[ca, -sa], [sa, ca]], np.float32)
                    Rb = np.array([[cb, -sb], [sb, cb]], np.float32)
                    mm = Ra @ m @ Rb.T
                    for (i, j, v, ok) in ((pa, pb, mm[0, 0], True), (pa, qb, mm[0, 1], rb), (qa, pb, mm[1, 0], ra),
                                          (qa, qb, mm[1, 1], ra and rb)):
                        if ok:
                            Anew[i, j] = Anew[j, i] = v
            A = Anew
        if not rotated:
            break
    W = np.eye(k, dtype=np.float32)
    for pairs in log:
        for (p, q, c, s, _) in pairs:
            if s != 0 and q < k:
                wp, wq = W[:, p].copy(), W[:, q].copy()
                W[:, p] = c * wp - s * wq
                W[:, q] = s * wp + c * wq
    return np.diag(A).astype(np.float64), W.astype(np.float64), len(log) // max(1, K - 1)


@pytest.mark.parametrize("k,spread", [(2, 3.0), (5, 4.0), (16, 6.0), (33, 5.0)])
def test_packed_jacobi_rounds_diagonalise(k, spread):
    """The one-pass block update of the packed Jacobi kernel, emulated in float32: W^T G W is diagonal
    to float accuracy, W orthonormal, and the Rayleigh quotients of W's columns (taken in double, as
    the library does next) match the spectrum to float accuracy relative to ||G||."""
    rng = np.random.default_rng(k)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    ev = 10.0 ** (-spread * rng.uniform(0, 1, k))
    G = (Q * ev) @ Q.T
    lam, W, sweeps = _packed_jacobi(G)
    assert sweeps < 30
    np.testing.assert_allclose(W.T @ W, np.eye(k), atol=2e-5 * k)
    rq = np.einsum("ij,ij->j", W, G @ W) / np.einsum("ij,ij->j", W, W)
    np.testing.assert_allclose(np.sort(rq)[::-1], np.sort(ev)[::-1], rtol=0, atol=1e-5 * ev.max())
    off = W.T @ G @ W - np.diag(np.diag(W.T @ G @ W))
    assert np.abs(off).max() <= 1e-5 * ev.max() * k
