"""Randomized Block Lanczos (Alg. 2) and its q = 1 range sketch, float64 (oracle; test infrastructure).

The paper runs Alg. 2 on A = Xbar, the d x n matrix whose i-th column is
n^{-1/2} x_i, so that A A^T = C (Sec. 5.3; the 1/n scaling printed in Alg. 3 is
read as n^{-1/2}, which makes sigma~_i^2 estimate the eigenvalues of C).  With
rows of X the examples, A = X^T / sqrt(n).
"""

import numpy as np

from . import streams


def test_matrix_gaussian(seed, n, k):
    """Pi ~ N(0,1)^{n x k} of Alg. 2 from the Gaussian Philox stream."""
    return streams.gaussian(seed, n, k)


def countsketch_rows(X, seed, s):
    """S X for the CountSketch S (s x n) with one nonzero sigma(i) at (h(i), i) per column:
    row h of S X is sum over {i : h(i) = h} of sigma(i) x_i.  Summed in row order."""
    X = np.asarray(X, np.float64)
    bucket, sign = streams.countsketch_hash(seed, X.shape[0], s)
    SX = np.zeros((s, X.shape[1]))
    for i in range(X.shape[0]):
        SX[bucket[i]] += sign[i] * X[i]
    return SX


def countsketch_matrix(seed, n, s):
    """The CountSketch as an explicit dense s x n matrix (for brute-force checks)."""
    bucket, sign = streams.countsketch_hash(seed, n, s)
    S = np.zeros((s, n))
    S[bucket, np.arange(n)] = sign
    return S


def range_sketch(X, k, seed, kind="gaussian", s=0, pi_bf16=False):
    """First Krylov block A Pi of Alg. 2, up to the scalar n^{-1/2}: Y = X^T Pi (d x k).

    kind = "gaussian":     Pi ~ N(0,1)^{n x k}.
    kind = "countsketch":  Pi = S^T G' with S an s x n CountSketch and G' ~ N(0,1)^{s x k},
                           i.e. Y = (S X)^T G'.  (Not in the paper: a cheaper
                           Gaussian-equivalent test matrix for the first pass.)
    """
    X = np.asarray(X, np.float64)
    if kind == "gaussian":
        Pi = test_matrix_gaussian(seed, X.shape[0], k)
        return X.T @ (streams.round_bf16(Pi) if pi_bf16 else Pi)
    if kind == "countsketch":
        return countsketch_rows(X, seed, s).T @ streams.gaussian(seed, s, k)
    raise ValueError(kind)


def krylov_blocks(X, Y0, q):
    """K = [A Pi, (A A^T) A Pi, ..., (A A^T)^{q-1} A Pi] of Alg. 2 with A A^T = C."""
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    blocks = [np.asarray(Y0, np.float64)]
    for _ in range(q - 1):
        blocks.append(X.T @ (X @ blocks[-1]) / n)
    return np.hstack(blocks)


def orthonormalize(K):
    """Q with orthonormal columns spanning K (Alg. 2, "orthonormalize"); Householder QR
    (library), with the column signs fixed so that diag(R) > 0, which makes Q unique."""
    Q, R = np.linalg.qr(np.asarray(K, np.float64))
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sgn


def ritz(X, Q, k):
    """Truncated SVD (Q^T A)_k = W~ Sigma~ V~^T and U~ = Q W~ (Alg. 2, last two steps).

    Returns U~ (d x k, the approximate leading eigenvectors of C) and sigma~^2
    (k values, descending).
    """
    X = np.asarray(X, np.float64)
    QtA = (X @ Q).T / np.sqrt(X.shape[0])          # Q^T A, k' x n
    W, s, _ = np.linalg.svd(QtA, full_matrices=False)
    return Q @ W[:, :k], s[:k] ** 2


def block_lanczos(X, k, seed, q=1, kind="gaussian", s=0, pi_bf16=False):
    """Alg. 2: returns (U~_k, sigma~^2).  q = 1 is the single-pass range sketch.  ``pi_bf16``: the
    Gaussian test matrix with its entries rounded to bfloat16 (the tensor-core sketch of bfloat16
    data draws the same Philox / Box-Muller values and rounds them)."""
    Y0 = range_sketch(X, k, seed, kind, s, pi_bf16)
    Q = orthonormalize(krylov_blocks(X, Y0, q))
    return ritz(X, Q, k)


def sym_eig_desc(G):
    """Eigen-decomposition of a symmetric matrix, eigenvalues descending (library routine)."""
    ev, W = np.linalg.eigh(np.asarray(G, np.float64))
    order = np.argsort(ev)[::-1]
    return ev[order], W[:, order]
