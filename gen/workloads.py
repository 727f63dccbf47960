"""The named synthetic workloads (inputs only; no sorting arithmetic).

The paper sorts "random uniformly drawn integers", the same set for every
algorithm (Section 4). The workloads below are seeded synthetic stand-ins of
that kind, plus the segmented, skewed and 64-bit families the library also
serves. No public dataset is involved. Seeds: 1 small uniform, 2 large uniform,
3 large 20-bit range, 4 segmented, 5 64-bit, 6 skewed; stream 0 carries keys.
"""
from __future__ import annotations

import numpy as np

from . import (gmm_u32, iota_u32, loguniform_lengths, lognormal_u32, uniform_u32, uniform_u64,
               zipf_u32)

SMALL_N = 65536          # small uniform u32 sort; BTN/OET take its first 1024 keys
SMALL_BTN_N = 1024
LARGE_N = 1 << 28        # large uniform u32 with payload = index
SEG_COUNT = 200_000      # segment lengths drawn before the cap
SEG_LO, SEG_HI = 2, 65536
SEG_CAP = 1 << 28        # total keys kept (longest prefix of segments under the cap)
SKEW_N = 1 << 28
WIDE_N = 1 << 27


def small_uniform(n: int = SMALL_N, seed: int = 1):
    """n u32 keys uniform on [0, 2^32), keys only."""
    return uniform_u32(n, 32, seed, 0)


def large_uniform(n: int = LARGE_N, bits: int = 32, seed: int = 2, payload: bool = True):
    """n u32 keys uniform on [0, 2^bits) and payload = index (or None)."""
    k = uniform_u32(n, bits, seed, 0)
    return k, (iota_u32(n) if payload else None)


def large_range20(n: int = LARGE_N, seed: int = 3, payload: bool = True):
    """n u32 keys uniform on [0, 2^20) with payload = index."""
    return large_uniform(n, 20, seed, payload)


def segment_offsets(seed: int = 4, nseg: int = SEG_COUNT, cap: int = SEG_CAP, lo: int = SEG_LO,
                    hi: int = SEG_HI):
    """CSR offsets (nseg_kept + 1, uint64) of log-uniform segment lengths.

    All nseg lengths are drawn; the longest prefix whose total stays <= cap is
    kept, and the realised segment count is len(offsets) - 1.
    """
    L = loguniform_lengths(nseg, lo, hi, seed, 1)
    c = np.cumsum(L, dtype=np.uint64)
    keep = int(np.searchsorted(c, np.uint64(cap), side="right"))
    off = np.zeros(keep + 1, np.uint64)
    off[1:] = c[:keep]
    return off


def segmented(seed: int = 4, nseg: int = SEG_COUNT, cap: int = SEG_CAP, payload: bool = True):
    """(keys, vals, offsets) for the batched segmented sort."""
    off = segment_offsets(seed, nseg, cap)
    n = int(off[-1])
    k = uniform_u32(n, 32, seed, 0)
    return k, (iota_u32(n) if payload else None), off


SKEW_KINDS = ("zipf", "lognormal", "gmm")


def skewed(kind: str, n: int = SKEW_N, seed: int = 6):
    """Skewed u32 keys: Zipf(1.1) hashed ranks, lognormal(20, 2) truncated, or a
    16-component Gaussian mixture (sigma 2^20) clipped."""
    if kind == "zipf":
        return zipf_u32(n, 1.1, seed, 10)
    if kind == "lognormal":
        return lognormal_u32(n, 20.0, 2.0, seed, 11)
    if kind == "gmm":
        return gmm_u32(n, 16, float(1 << 20), seed, 12)
    raise ValueError(kind)


def wide_u64(n: int = WIDE_N, bits: int = 64, seed: int = 5, payload: bool = True):
    """n u64 keys uniform on [0, 2^bits) with payload = index."""
    k = uniform_u64(n, bits, seed, 0 if bits == 64 else 2)
    return k, (iota_u32(n) if payload else None)
