"""Philox4x32-10 words from triton's own implementation, run by triton's CPU interpreter.

Used only as an independent library implementation to pin the oracle's generator.
"""
import os

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402



@triton.jit
def _kern(c_ptr, out_ptr, seed, NB: tl.constexpr):
    o = tl.arange(0, NB)
    c0 = tl.load(c_ptr + o * 4 + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + o * 4 + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + o * 4 + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + o * 4 + 3).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + o * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 3, d.to(tl.int32, bitcast=True))


def philox_words(counters, seed):
    nb = counters.shape[0]
    c = torch.from_numpy(counters.astype(np.uint32).view(np.int32).copy())
    out = torch.zeros(nb * 4, dtype=torch.int32)
    _kern[(1,)](c, out, seed, nb)
    return out.numpy().view(np.uint32).reshape(nb, 4)
