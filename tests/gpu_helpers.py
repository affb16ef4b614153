"""Helpers for the GPU tests: device copies with the 16-byte row stride the C ABI requires."""

import torch


def cuda_rows(t):
    """CUDA copy of a 2-D tensor whose row stride is padded to a multiple of 16 bytes."""
    n, d = t.shape
    es = t.element_size()
    ld = ((d * es + 15) // 16 * 16) // es
    buf = torch.zeros(n, ld, dtype=t.dtype, device="cuda")
    buf[:, :d] = t.to("cuda")
    return buf[:, :d]
