"""Pins for oracle.sketch (Alg. 2): brute force, exact recovery, Rayleigh-Ritz facts."""

import numpy as np
import pytest

from oracle import ridge, sketch, streams
from paper_1602_02350_gb300 import synth


def _data(n, d, alpha=1.5, seed=3):
    X, y, _ = synth.problem(n, d, np.arange(1, d + 1) ** -alpha, 0.1, seed)
    return X.numpy(), y.numpy()


def test_countsketch_rows_equals_dense_sketch_product():
    X, _ = _data(300, 10)
    SX = sketch.countsketch_rows(X, 17, 32)
    S = sketch.countsketch_matrix(17, 300, 32)
    np.testing.assert_allclose(SX, S @ X, rtol=1e-13, atol=1e-13)
    # a CountSketch has exactly one +-1 per column, so S^T S has unit diagonal
    assert np.all(np.diag(S.T @ S) == 1.0)


def test_range_sketch_of_identity_is_the_test_matrix():
    Y = sketch.range_sketch(np.eye(40), 6, 5)
    np.testing.assert_array_equal(Y, streams.gaussian(5, 40, 6))
    # CountSketch form: Pi = S^T G'
    Yc = sketch.range_sketch(np.eye(40), 6, 5, kind="countsketch", s=8)
    S = sketch.countsketch_matrix(5, 40, 8)
    np.testing.assert_allclose(Yc, S.T @ streams.gaussian(5, 8, 6), rtol=1e-14)


def test_orthonormalize_gives_qr_factor():
    Y = synth.random_matrix(50, 7, 2)
    Q = sketch.orthonormalize(Y)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-13)
    R = Q.T @ Y
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-12)     # upper triangular
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q @ R, Y, rtol=1e-12, atol=1e-12)


def test_exact_recovery_when_rank_at_most_k():
    # X of rank 4 in R^12: the sketch with k = 4 recovers C's spectrum and eigenspace exactly
    rng = np.random.default_rng(0)
    X = rng.standard_normal((200, 4)) @ rng.standard_normal((4, 12))
    U, s2 = sketch.block_lanczos(X, 4, seed=9)
    C = ridge.correlation(X)
    ev, W = np.linalg.eigh(C)
    np.testing.assert_allclose(s2, ev[::-1][:4], rtol=1e-10)
    P = W[:, -4:] @ W[:, -4:].T
    np.testing.assert_allclose(U @ U.T, P, atol=1e-10)


def test_ritz_values_interlace_and_match_projected_matrix():
    X, _ = _data(400, 30)
    U, s2 = sketch.block_lanczos(X, 5, seed=4)
    C = ridge.correlation(X)
    lam = np.sort(np.linalg.eigvalsh(C))[::-1]
    # Cauchy interlacing for the Rayleigh-Ritz values of a k-dimensional subspace
    assert np.all(s2 <= lam[:5] * (1 + 1e-12))
    Q = sketch.orthonormalize(sketch.range_sketch(X, 5, 4))
    ritz = np.sort(np.linalg.eigvalsh(Q.T @ C @ Q))[::-1]
    np.testing.assert_allclose(s2, ritz, rtol=1e-10)
    # U~ are eigenvectors of the projected problem: U^T C U = diag(s2)
    np.testing.assert_allclose(U.T @ C @ U, np.diag(s2), atol=1e-12 * lam[0])
    np.testing.assert_allclose(U.T @ U, np.eye(5), atol=1e-12)


def test_block_lanczos_per_vector_bound_soft():
    """Thm 3's per-vector bound |sigma~_i^2 - sigma_i^2| <= eps' sigma_{k+1}^2 with eps' = 1/2
    holds with probability 9/10 for q = Theta(log n); checked over seeds."""
    X, _ = _data(800, 60, alpha=1.0, seed=8)
    lam = np.sort(np.linalg.eigvalsh(ridge.correlation(X)))[::-1]
    k, ok = 6, 0
    for seed in range(10):
        _, s2 = sketch.block_lanczos(X, k, seed=seed, q=6)
        ok += np.all(np.abs(s2 - lam[:k]) <= 0.5 * lam[k])
    assert ok >= 9


def test_more_krylov_blocks_never_hurt_the_ritz_values():
    X, _ = _data(500, 40, alpha=1.0, seed=12)
    _, s1 = sketch.block_lanczos(X, 5, seed=1, q=1)
    _, s3 = sketch.block_lanczos(X, 5, seed=1, q=3)
    # the q = 3 Krylov space contains the q = 1 space: Ritz values can only grow
    assert np.all(s3 >= s1 * (1 - 1e-12))


def test_sym_eig_desc_reconstructs():
    G = synth.random_symmetric(9, 1)
    ev, W = sketch.sym_eig_desc(G)
    assert np.all(np.diff(ev) <= 0)
    np.testing.assert_allclose((W * ev) @ W.T, G, atol=1e-14)
    np.testing.assert_allclose(W.T @ W, np.eye(9), atol=1e-13)


def test_countsketch_mode_is_unbiased_for_the_gram():
    # E[S^T S] = I, so (S X)^T (S X) estimates X^T X: average over seeds
    X, _ = _data(256, 5)
    acc = np.zeros((5, 5))
    for seed in range(200):
        SX = sketch.countsketch_rows(X, seed, 16)
        acc += SX.T @ SX
    rel = np.linalg.norm(acc / 200 - X.T @ X) / np.linalg.norm(X.T @ X)
    assert rel < 0.05
    with pytest.raises(ValueError):
        sketch.range_sketch(X, 2, 0, kind="nope")
