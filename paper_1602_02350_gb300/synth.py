"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws inputs.  It holds none of the method's arithmetic, so it
is the one piece of code that both the CUDA path and the CPU oracle are fed
from.  Rows follow x_i = Q diag(sqrt(s)) g_i with g_i ~ N(0, I) and Q a
Haar-random orthogonal basis, so the correlation matrix C = X^T X / n has
expected eigenvalues s_j (power-law spectra as in the paper's synthetic
experiments, Sec. 6).  Labels are y = X w_gen + noise * N(0, 1) with
w_gen ~ N(0, 1/d); w_gen is the generating vector, not the ridge minimiser.
"""

from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class Config:
    """One synthetic workload: shapes, spectrum, noise, lambda, sketch and SVRG settings."""
    name: str
    n: int
    d: int
    alpha: float            # s_j = j^-alpha
    noise: float
    lam: float
    k: int
    kind: str = "gaussian"  # or "countsketch"
    s: int = 0              # CountSketch rows
    boost_top: int = 0      # number of leading directions multiplied by boost
    boost: float = 1.0
    dtype: str = "f32"
    seed_data: int = 1000
    seed_sketch: int = 2000
    seed_svrg: int = 3000
    epochs: int = 20
    m: int = 0              # 0 = theory default ceil(beta^ / lam)
    eta_mult: float = 0.1   # eta = eta_mult / beta^ (0.1 is the Thm 2 value)
    extra: dict = field(default_factory=dict)

    def spectrum(self):
        j = np.arange(1, self.d + 1, dtype=np.float64)
        s = j ** (-self.alpha)
        if self.boost_top:
            s[: self.boost_top] *= self.boost
        return s


# The paper's sizes are too large for a float64 check on every commit; these are
# the workloads the library is measured and checked on (seeds 1000+i, 2000+i, 3000+i).
CONFIGS = {
    # plain method, FP64 against the oracle
    "fp64_n4096_d256": Config("fp64_n4096_d256", 4096, 256, 1.5, 0.1, 1e-4, 16, dtype="f64",
                              seed_data=1000, seed_sketch=2000, seed_svrg=3000, epochs=20, m=8192,
                              eta_mult=1.0),
    # plain method FP32, CountSketch (s = 4096) then Gaussian, run to 1e-6
    "fp32_n65536_d1024": Config("fp32_n65536_d1024", 65536, 1024, 2.0, 0.05, 1e-5, 64,
                                kind="countsketch", s=4096, dtype="f32",
                                seed_data=1001, seed_sketch=2001, seed_svrg=3001, epochs=30),
    # BF16 storage with FP32 refinement
    "bf16_n1048576_d4096": Config("bf16_n1048576_d4096", 1 << 20, 4096, 1.2, 0.05, 1e-6, 256,
                                  boost_top=20, boost=100.0, dtype="bf16",
                                  seed_data=1002, seed_sketch=2002, seed_svrg=3002, epochs=30),
}


def haar_orthogonal(d, seed):
    """Haar-distributed d x d orthogonal matrix: QR of a Gaussian matrix with the signs of
    diag(R) moved into Q (Mezzadri 2007)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))


def problem(n, d, spectrum, noise, seed, device="cpu", dtype=torch.float64):
    """X (n x d), y (n), w_gen (d) as torch tensors on ``device`` (rows generated in chunks).

    On CPU the Gaussian draws come from numpy's PCG64; on CUDA from torch's CUDA
    generator (faster for large n).  Either way the same call returns the same data.
    """
    spectrum = np.asarray(spectrum, np.float64)
    Q = torch.from_numpy(haar_orthogonal(d, seed + 7))
    rng = np.random.default_rng(seed)
    w_gen = torch.from_numpy(rng.standard_normal(d) / np.sqrt(d))
    dev = torch.device(device)
    scale = torch.from_numpy(np.sqrt(spectrum))
    if dev.type == "cuda":
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        Qs = (Q * scale[None, :]).to(dev, torch.float32).T.contiguous()   # diag(sqrt s) Q^T
        X = torch.empty((n, d), dtype=dtype, device=dev)
        y = torch.empty(n, dtype=torch.float64, device=dev)
        wg = w_gen.to(dev)
        chunk = max(1, (1 << 26) // d)
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            G = torch.randn((r1 - r0, d), generator=gen, device=dev, dtype=torch.float32)
            xb = torch.matmul(G, Qs)
            X[r0:r1] = xb.to(dtype)
            eps = torch.randn(r1 - r0, generator=gen, device=dev, dtype=torch.float32)
            y[r0:r1] = X[r0:r1].double() @ wg + noise * eps.double()
        return X, y, w_gen.to(dev)
    Qs = (Q * scale[None, :]).T.contiguous()
    G = torch.from_numpy(rng.standard_normal((n, d)))
    Xd = G @ Qs
    X = Xd.to(dtype)
    eps = torch.from_numpy(rng.standard_normal(n))
    y = X.double() @ w_gen + noise * eps
    return X, y, w_gen


def spectrum_problem(n, d, decay, noise, seed, device="cuda", dtype=torch.float32):
    """The synthetic data of the paper's Sec. 6 at n x d: a d x n matrix with uniformly random singular
    vectors and q-th singular value q^-decay (decay 1: linear, 2: quadratic), examples (its columns)
    normalised to unit norm, labels y_i = w_gen^T x_i + noise N(0, 1) with w_gen ~ N(0, I_d).
    Rows of the returned X are the examples: X = V diag(s) U^T with U (d x d) and V (n x d) orthonormal
    (QR of seeded Gaussians, signs fixed), then each row scaled to norm 1."""
    dev = torch.device(device)
    U = torch.from_numpy(haar_orthogonal(d, seed + 11))
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    G = torch.randn((n, d), generator=gen, device=dev, dtype=torch.float64)
    Vq, R = torch.linalg.qr(G)
    Vq = Vq * torch.sign(torch.diagonal(R))[None, :]
    del G, R
    s = torch.arange(1, d + 1, dtype=torch.float64, device=dev) ** (-float(decay))
    X = (Vq * s[None, :]) @ U.to(dev).T
    del Vq
    X = X / X.norm(dim=1, keepdim=True)
    rng = np.random.default_rng(seed)
    w_gen = torch.from_numpy(rng.standard_normal(d)).to(dev)
    eps = torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    Xs = X.to(dtype)
    y = Xs.double() @ w_gen + noise * eps
    return Xs.contiguous(), y, w_gen


def config_problem(cfg, device="cpu", dtype=None):
    """The data of a named configuration."""
    if dtype is None:
        dtype = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[cfg.dtype]
    return problem(cfg.n, cfg.d, cfg.spectrum(), cfg.noise, cfg.seed_data, device, dtype)


# --- small random inputs for per-step parity tests -------------------------------------------

def random_orthonormal(d, k, seed):
    """d x k matrix with orthonormal columns (first k columns of a Haar matrix)."""
    return haar_orthogonal(d, seed)[:, :k].copy()


def random_sigma2(k, seed, lo=1e-4, hi=1.0):
    """k positive values, descending, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), k)))[::-1].copy()


def random_matrix(rows, cols, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((rows, cols))


def random_vector(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(n)


def random_symmetric(k, seed, spread=6.0):
    """Symmetric positive semi-definite k x k matrix with eigenvalues spread over 10^spread."""
    rng = np.random.default_rng(seed)
    Q = haar_orthogonal(k, seed + 1)
    ev = 10.0 ** (-spread * rng.uniform(0, 1, k))
    return (Q * ev) @ Q.T


def random_weights(N, seed, hi=1 << 24):
    """Positive integer sampling weights in [1, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(1, hi + 1, N, dtype=np.int64).astype(np.uint32)


def random_indices(N, m, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, N, m, dtype=np.int64)


def random_positive(m, seed, lo=0.5, hi=2.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, m)


# --- proposal network ---------------------------------------------------------------------------

MLP_SHAPES = [(128, 67), (128,), (128, 128), (128,), (3, 128), (3,)]


def mlp_init(seed):
    """Flat float64 parameter vector of the 67 -> 128 -> 128 -> 3 network: weights drawn
    N(0, 2 / fan_in) (He et al., 2015), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in MLP_SHAPES:
        parts.append(rng.standard_normal(s).ravel() * np.sqrt(2.0 / s[1]) if len(s) == 2 else np.zeros(s))
    return np.concatenate(parts)
