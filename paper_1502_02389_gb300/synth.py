"""Seeded synthetic inputs for the asum / dot / scal / gemv workloads.

This module only draws and stores inputs; it holds none of the arithmetic of
the map/reduce programs.  Both the GPU path and the CPU oracle receive the
arrays it returns.  All draws use NumPy ``Generator(PCG64(seed))`` in
float64, cast with round-to-nearest-even to the storage type; within one
workload the draw order is x, then y, then A, then masks.

Workloads (sizes of the paper's BLAS experiments, Sec. 7.2, scaled to a
GB300):
  asum_small     n = 2^20,  x ~ U(-1, 1),                 seed 0
  dot_scal       n = 2^26,  x, y ~ N(0, 1), alpha = 1.5,  seed 1
  gemv           A (M x N) and x ~ U(-1, 1), y ~ U(-1, 1), alpha = 1,
                 beta = 0.5, seed 2; M x N = 8192 x 8192 or 65536 x 1024
  mixed          n = 2^28, N(0, 1) with 1 % of entries scaled by 1e3,
                 stored as bf16 or as fp8-e4m3 with one fp32 scale per 4096
                 consecutive elements, seed 4
"""
from __future__ import annotations

import numpy as np

FP8_BLOCK = 4096
FP8_MAX = 448.0


def generator(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def asum_small(n: int = 1 << 20, seed: int = 0) -> np.ndarray:
    g = generator(seed)
    return g.uniform(-1.0, 1.0, n).astype(np.float32)


def dot_scal(n: int = 1 << 26, seed: int = 1):
    g = generator(seed)
    x = g.standard_normal(n).astype(np.float32)
    y = g.standard_normal(n).astype(np.float32)
    return x, y, np.float32(1.5)


def gemv(M: int, N: int, seed: int = 2):
    g = generator(seed)
    x = g.uniform(-1.0, 1.0, N).astype(np.float32)
    y = g.uniform(-1.0, 1.0, M).astype(np.float32)
    A = g.uniform(-1.0, 1.0, (M, N)).astype(np.float32)
    return A, x, y, np.float32(1.0), np.float32(0.5)


def mixed_values(n: int = 1 << 28, seed: int = 4, two: bool = True):
    """FP64 draws x (and y) with 1 % of the entries scaled by 1e3."""
    g = generator(seed)
    x = g.standard_normal(n)
    y = g.standard_normal(n) if two else None
    mx = g.random(n) < 0.01
    x[mx] *= 1e3
    if two:
        my = g.random(n) < 0.01
        y[my] *= 1e3
    return x, y


# ---------------------------------------------------------------------------
# storage encodings (round to nearest, ties to even, from FP64)
# ---------------------------------------------------------------------------
def _round_to_bits(v: np.ndarray, sig_bits: int, min_exp: int) -> np.ndarray:
    """Round v to ``sig_bits`` significant bits, with a quantum no smaller
    than 2^(min_exp - sig_bits + 1) (gradual underflow), ties to even."""
    v = np.asarray(v, np.float64)
    _, e = np.frexp(v)                    # v = m * 2^e, 0.5 <= |m| < 1
    lead = np.maximum(e - 1, min_exp)     # exponent of the leading bit
    quantum = np.exp2((lead - (sig_bits - 1)).astype(np.float64))
    return np.rint(v / quantum) * quantum  # np.rint rounds half to even


def encode_bf16(v) -> np.ndarray:
    """FP64 -> bf16 bit patterns (uint16), RNE, one rounding."""
    r = _round_to_bits(v, 8, -126)
    return (r.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def encode_e4m3(v) -> np.ndarray:
    """FP64 (already scaled) -> fp8-e4m3 bit patterns, RNE, saturating to
    +-448."""
    v = np.asarray(v, np.float64)
    r = _round_to_bits(v, 4, -6)
    r = np.clip(r, -FP8_MAX, FP8_MAX)
    a = np.abs(r)
    sign = (np.signbit(r)).astype(np.uint8) << 7
    _, e = np.frexp(np.where(a == 0, 1.0, a))
    lead = e - 1
    normal = a >= 2.0 ** -6
    exp_field = np.where(normal, lead + 7, 0)
    frac = np.where(normal, a / np.exp2(lead.astype(np.float64)) - 1.0, a / 2.0 ** -6)
    frac_field = np.rint(frac * 8.0).astype(np.int64)
    out = sign | (exp_field.astype(np.uint8) << 3) | frac_field.astype(np.uint8)
    return np.where(a == 0, sign, out).astype(np.uint8)


def block_scales(v, block: int = FP8_BLOCK) -> np.ndarray:
    """One fp32 scale per block: amax / 448 (1 for an all-zero block)."""
    v = np.asarray(v, np.float64)
    nb = (v.size + block - 1) // block
    pad = np.zeros(nb * block)
    pad[: v.size] = np.abs(v)
    amax = pad.reshape(nb, block).max(axis=1)
    s = (amax / FP8_MAX).astype(np.float32)
    return np.where(amax == 0, np.float32(1.0), s).astype(np.float32)


def encode_fp8_blocks(v, block: int = FP8_BLOCK):
    """FP64 values -> (e4m3 bit patterns, fp32 scales per block)."""
    v = np.asarray(v, np.float64)
    s = block_scales(v, block)
    blk = np.arange(v.size) // block
    q = encode_e4m3(v / s[blk].astype(np.float64))
    return q, s
