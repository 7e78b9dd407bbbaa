"""Mixed-precision asum and dot: exact decoding of the stored values and the
FP64 definitions over them.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

Storage formats (IEEE-style bit layouts, decoded here from their
definitions; no lookup table is shared with the GPU path):
  * bf16: sign 1, exponent 8 (bias 127), fraction 7 -- the upper 16 bits of
    an IEEE binary32 value.
  * fp8-e4m3 (OCP 8-bit floating point, E4M3): sign 1, exponent 4 (bias 7),
    fraction 3; exponent field 0 encodes subnormals f/8 * 2^-6; the pattern
    S.1111.111 is NaN; there are no infinities; the largest finite value is
    1.75 * 2^8 = 448.  An fp8 vector carries one fp32 scale s_b per block of
    4096 consecutive elements (the last block may be shorter); the stored
    value of element i is q_i * s_{i // 4096}.

Every decoded value (and q_i * s_b) is exact in FP64, so the definitions
below are the plain programs of Fig. 5 on exactly promoted stored values:
asum = reduce(add, 0) . map(abs), dot = reduce(add, 0) . map(mult) . zip.
"""
from __future__ import annotations

import numpy as np

from . import blas

FP8_BLOCK = 4096


def decode_bf16(bits) -> np.ndarray:
    """uint16 bit patterns -> FP64 values (exact)."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def decode_e4m3(bits) -> np.ndarray:
    """uint8 bit patterns -> FP64 values (exact), from the E4M3 definition."""
    b = np.asarray(bits, dtype=np.uint8).astype(np.int64)
    sign = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    f = b & 0x7
    normal = sign * (1.0 + f / 8.0) * np.exp2(e - 7.0)
    sub = sign * (f / 8.0) * 2.0 ** -6
    val = np.where(e == 0, sub, normal)
    return np.where((e == 0xF) & (f == 0x7), np.nan, val)


def stored_values(dtype: str, data, scales=None) -> np.ndarray:
    """The FP64 values a stored vector represents."""
    if dtype == "f32":
        return np.asarray(data, np.float32).astype(np.float64)
    if dtype == "bf16":
        return decode_bf16(data)
    if dtype == "fp8":
        q = decode_e4m3(data)
        s = np.asarray(scales, np.float32).astype(np.float64)
        blk = np.arange(q.size) // FP8_BLOCK
        return q * s[blk]
    raise ValueError(dtype)


def asum(dtype: str, data, scales=None) -> float:
    return blas.asum(stored_values(dtype, data, scales))


def dot(dtype: str, x, xs, y, ys) -> float:
    return blas.dot(stored_values(dtype, x, xs), stored_values(dtype, y, ys))
