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
  batch          20,000 ops, op uniform over {asum, dot, gemv}, vector
                 lengths round(2^U(8, 22)), gemv M, N = round(2^U(6, 12))
                 independently (PCG64 seed 3); every array a disjoint,
                 256-byte aligned slice of one pool (about 60 GB) whose values
                 are N(0, 1), drawn on the device by torch's generator seeded
                 3 (drawing 15 G values on the host would take minutes); gemv
                 alpha = 1, beta = 0.5
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


def gemv_t(M: int, N: int, seed: int = 5):
    """y <- alpha A^T x + beta y inputs: A (M x N), x (M), y (N), all
    U(-1, 1); alpha = 1, beta = 0.5."""
    g = generator(seed)
    x = g.uniform(-1.0, 1.0, M).astype(np.float32)
    y = g.uniform(-1.0, 1.0, N).astype(np.float32)
    A = g.uniform(-1.0, 1.0, (M, N)).astype(np.float32)
    return A, x, y, np.float32(1.0), np.float32(0.5)


# BlackScholes options (Fig. 6 maps over the stock prices only, so the other
# model inputs are shared constants)
BS_STRIKE, BS_RATE, BS_VOL, BS_YEARS = 20.0, 0.02, 0.30, 1.0


def stock_prices(n: int, seed: int = 6) -> np.ndarray:
    """Stock prices U(5, 30)."""
    return generator(seed).uniform(5.0, 30.0, n).astype(np.float32)


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


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------
ASUM, DOT, GEMV = 0, 1, 3   # op ids of the library's C-ABI


def batch_ops(count: int = 20000, seed: int = 3, lo: float = 8, hi: float = 22,
              mlo: float = 6, mhi: float = 12):
    """Op types and sizes of the batched workload."""
    g = generator(seed)
    kind = g.integers(0, 3, count)
    n = np.rint(2.0 ** g.uniform(lo, hi, count)).astype(np.int64)
    M = np.rint(2.0 ** g.uniform(mlo, mhi, count)).astype(np.int64)
    N = np.rint(2.0 ** g.uniform(mlo, mhi, count)).astype(np.int64)
    ops = []
    for i in range(count):
        op = (ASUM, DOT, GEMV)[int(kind[i])]
        if op == GEMV:
            ops.append({"op": op, "n": 0, "M": int(M[i]), "N": int(N[i])})
        else:
            ops.append({"op": op, "n": int(n[i]), "M": 0, "N": 0})
    return ops


def batch_layout(ops, align_elems: int = 64):
    """Disjoint, 256-byte aligned element offsets into one fp32 pool:
    per op {'x', 'y', 'A', 'out'} (absent arrays omitted); returns the
    offsets and the pool length in elements."""
    off = 0
    lay = []

    def take(count):
        nonlocal off
        o = off
        off += (max(count, 1) + align_elems - 1) // align_elems * align_elems
        return o

    for d in ops:
        e = {}
        if d["op"] == GEMV:
            e["A"] = take(d["M"] * d["N"])
            e["x"] = take(d["N"])
            e["out"] = take(d["M"])
        else:
            e["x"] = take(d["n"])
            if d["op"] == DOT:
                e["y"] = take(d["n"])
            e["out"] = take(1)
        lay.append(e)
    return lay, off
