"""The four BLAS programs of arXiv 1502.02389, Fig. 5, written in the
high-level patterns and evaluated by the FP64 interpreter.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

    scal(a, x)          = map(mult(a), x)
    asum(x)             = reduce(add, 0) . map(abs, x)
    dot(x, y)           = reduce(add, 0) . map(mult) . zip(x, y)
    gemv(A, x, y, a, b) : z = map(scal(a) . dot(x), A)
                          map(add) . zip(z, scal(b, y))

gemv computes y = a*A*x + b*y "as defined by the BLAS library" (Sec. 5.1).
Two readings are taken where Fig. 5 leaves room:
  * map(scal(a) . dot(x), A) yields one length-1 array per row (every value
    is an array, Sec. 3), so z is that result joined to length M before the
    zip with y;
  * with b = 0 the BLAS definition does not read y, so y' = a*A*x and a NaN
    in y does not propagate.

The parity tolerance for an fp32 result r against the FP64 value v of a sum
of terms t_i is |r - v| <= 4 * 2^-24 * max(1, ceil(log2 n)) * sum|t_i|
(u = 2^-24 is the unit roundoff of fp32).
"""
from __future__ import annotations

import math

import numpy as np

from .patterns import (C, Join, Map, Reduce, ReorderStride, Split, Zip, ZipWith, abs_,
                       add, evaluate, mult, mult_by, sqrt64, square)

U_FP32 = 2.0 ** -24


def scal_expr(a):
    return Map(mult_by(a))


def asum_expr():
    return C(Reduce(add, 0), Map(abs_))


def dot_expr():
    return C(Reduce(add, 0), Map(mult), Zip())


def gemv_z_expr(a):
    """z = join . map(scal(a) . dot(x), A); dot(x) zips the captured x with
    each row of A."""
    dot_x = C(Reduce(add, 0), Map(mult), ZipWith("x"))
    return C(Join(), Map(C(scal_expr(a), dot_x)))


def gemv_y_expr():
    """y' = map(add) . zip(z, scal(b, y))."""
    return C(Map(add), Zip())


# ---------------------------------------------------------------------------
# user-function programs in the same style (the code generator only knows
# reduce-seq and the maps; any user functions plug in, Sec. 4.2 "Reduction")
#   nrm2(x)       = map(sqrt) . reduce(add, 0) . map(square, x)
#   sum(x)        = reduce(add, 0)(x)
#   axpy(a, x, y) = map(add) . zip(map(mult(a), x), y)
# ---------------------------------------------------------------------------
def nrm2_expr():
    return C(Map(sqrt64), Reduce(add, 0), Map(square))


def sum_expr():
    return Reduce(add, 0)


def axpy_expr():
    """Applied to the pair (scal(a, x), y)."""
    return C(Map(add), Zip())


def transpose_expr(M: int, N: int):
    """The columns of a row-major M x N matrix as rows: split^M .
    reorder-stride^N . join (Sec. 3.2: out[i] = in[i/n + s*(i mod n)] with
    s = N, n = M reads element (i mod M, i / M))."""
    return C(Split(M), ReorderStride(s=N), Join())


def gemv_t(A, x, y, alpha, beta, mode="f64"):
    """y' = alpha * A^T x + beta * y: the gemv program over the transposed
    view of A (x has M entries, y has N)."""
    A, x, y = np.asarray(A), np.asarray(x), np.asarray(y)
    M, N = A.shape
    if N == 0:
        return np.zeros(0)
    if M == 0:
        z = np.zeros(N)
    else:
        z = evaluate(C(gemv_z_expr(alpha), transpose_expr(M, N)), A, mode, env={"x": x})
    if beta == 0:
        return np.asarray(z, dtype=np.float64)
    return evaluate(gemv_y_expr(), (z, scal(beta, y, mode)), mode)


def nrm2(x, mode="f64") -> float:
    x = np.asarray(x)
    if x.size == 0:
        return 0.0
    return float(evaluate(nrm2_expr(), x, mode)[0])


def sum_(x, mode="f64") -> float:
    x = np.asarray(x)
    if x.size == 0:
        return 0.0
    return float(evaluate(sum_expr(), x, mode)[0])


def axpy(a, x, y, mode="f64"):
    x, y = np.asarray(x), np.asarray(y)
    return evaluate(axpy_expr(), (scal(a, x, mode), y), mode)


def asum_exact(x) -> float:
    """sum |x_i|, correctly rounded to FP64 (math.fsum)."""
    return math.fsum(np.abs(np.asarray(x, np.float64)))


def dot_exact(x, y) -> float:
    """sum x_i y_i, correctly rounded to FP64: the product of two fp32
    values is exact in FP64 (24 + 24 significant bits), and math.fsum adds
    the exact products with a single final rounding."""
    return math.fsum(np.asarray(x, np.float64) * np.asarray(y, np.float64))


def compensated_tolerance(value: float, sum_abs_terms: float, m: int) -> float:
    """Bound for a compensated sum: every term added with TwoSum into one of
    several (sum, compensation) pairs, at most m terms per pair, pairs merged
    with TwoSum, the result rounded once to fp32.  The compensated sum of m
    terms is within u|s| + gamma_m^2 sum|t| of the exact s (Ogita, Rump and
    Oishi 2005, Sum2; gamma_m ~ m u); the fp32 rounding adds u|s|.  With a
    factor 2 on the second-order term for the merges:
    2 u |v| + 2 (m u)^2 sum|t|."""
    return 2 * U_FP32 * abs(value) + 2 * (m * U_FP32) ** 2 * float(sum_abs_terms)


def nrm2_tolerance(n: int, sum_sq: float) -> float:
    """nrm2 = sqrt(S) with S = sum x_i^2 (all terms >= 0, so sum|terms| = S).
    An error e <= 4 u ceil(log2 n) S in S moves the root by
    e / (sqrt(S') + sqrt(S)) <= e / sqrt(S) = 4 u ceil(log2 n) sqrt(S); the
    final rounding to fp32 adds at most u sqrt(S') (bounded by 2 u sqrt(S)):
    (4 ceil(log2 n) + 2) u sqrt(S)."""
    return (4 * depth(n) + 2) * U_FP32 * math.sqrt(float(sum_sq))


def scal(a, x, mode="f64"):
    return evaluate(scal_expr(a), np.asarray(x), mode)


def asum(x, mode="f64") -> float:
    x = np.asarray(x)
    if x.size == 0:
        return 0.0  # reduce of an empty array is z (Table 1; Sec. 3.2)
    return float(evaluate(asum_expr(), x, mode)[0])


def dot(x, y, mode="f64") -> float:
    x, y = np.asarray(x), np.asarray(y)
    if x.size == 0:
        return 0.0
    return float(evaluate(dot_expr(), (x, y), mode)[0])


def gemv(A, x, y, alpha, beta, mode="f64"):
    """y' = alpha*A*x + beta*y (row-major A of shape (M, N))."""
    A, x, y = np.asarray(A), np.asarray(x), np.asarray(y)
    M, N = A.shape
    if M == 0:
        return np.zeros(0)
    if N == 0:
        z = np.zeros(M)
    else:
        z = evaluate(gemv_z_expr(alpha), A, mode, env={"x": x})
    if beta == 0:
        return np.asarray(z, dtype=np.float64)
    by = scal(beta, y, mode)
    return evaluate(gemv_y_expr(), (z, by), mode)


# ---------------------------------------------------------------------------
# tolerance
# ---------------------------------------------------------------------------
def depth(n: int) -> int:
    return max(1, math.ceil(math.log2(n))) if n > 1 else 1


def tolerance(n: int, sum_abs_terms: float) -> float:
    """4 * u_fp32 * max(1, ceil(log2 n)) * sum|terms|."""
    return 4.0 * U_FP32 * depth(n) * float(sum_abs_terms)


def asum_terms(x) -> float:
    return float(np.sum(np.abs(np.asarray(x, np.float64))))


def dot_terms(x, y) -> float:
    return float(np.sum(np.abs(np.asarray(x, np.float64) * np.asarray(y, np.float64))))


def gemv_row_terms(A, x, y, alpha, beta):
    """|alpha| * sum_j |A_ij x_j| + |beta * y_i| per row."""
    A = np.asarray(A, np.float64)
    x = np.asarray(x, np.float64)
    t = abs(alpha) * (np.abs(A) @ np.abs(x))
    if beta != 0:
        t = t + np.abs(beta * np.asarray(y, np.float64))
    return t
