"""Philox4x32-10 and Box-Muller normals, from their published definitions.

Philox: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (2011).  Ten rounds of two 32x32->64-bit
multiplies; the key is bumped by the Weyl constants between rounds.
Box-Muller: G. E. P. Box, M. E. Muller, Ann. Math. Stat. 29 (1958) 610.

Counter layout (shared *definition*, written independently on the CUDA side):
key = (seed & 0xffffffff, seed >> 32); counter = (element, step_lo, step_hi, tag).
Tags: 1 = initial mode positions, 2 = initial momenta, 3 = O-step noise,
4 = adQTB white noise.
"""
from __future__ import annotations

import numpy as np

MASK = np.uint64(0xFFFFFFFF)
M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)

TAG_INIT_Q = 1
TAG_INIT_P = 2
TAG_OSTEP = 3
TAG_QTB_WHITE = 4


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr: uint (...,4), key: uint (...,2) -> uint32 (...,4)."""
    ctr = np.asarray(ctr, dtype=np.uint64) & MASK
    key = np.asarray(key, dtype=np.uint64) & MASK
    c0, c1, c2, c3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0, k1 = np.broadcast_to(key[..., 0], c0.shape), np.broadcast_to(key[..., 1], c0.shape)
    for r in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def uniform53(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """Uniform in (0,1): k = (hi>>5)*2^26 + (lo>>6) (53 bits), u = (k + 1/2) * 2^-53."""
    k = (hi.astype(np.uint64) >> np.uint64(5)) * np.uint64(1 << 26) + (lo.astype(np.uint64) >> np.uint64(6))
    return (k.astype(np.float64) + 0.5) * 2.0 ** -53


def normals(seed: int, element: np.ndarray, step: int | np.ndarray, tag: int, which: int | np.ndarray = 0) -> np.ndarray:
    """Standard normal for each element at a step: Box-Muller on one Philox draw.

    which = 0 takes r*cos(2*pi*u2), which = 1 takes r*sin(2*pi*u2).
    """
    element = np.asarray(element, dtype=np.uint64)
    step = np.asarray(step, dtype=np.uint64)
    shape = np.broadcast_shapes(element.shape, step.shape)
    ctr = np.empty(shape + (4,), dtype=np.uint64)
    ctr[..., 0] = element & MASK
    ctr[..., 1] = step & MASK
    ctr[..., 2] = step >> np.uint64(32)
    ctr[..., 3] = tag
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    x = philox4x32_10(ctr, key)
    u1 = uniform53(x[..., 0], x[..., 1])
    u2 = uniform53(x[..., 2], x[..., 3])
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    which = np.asarray(which)
    return np.where(which == 0, r * np.cos(theta), r * np.sin(theta))
