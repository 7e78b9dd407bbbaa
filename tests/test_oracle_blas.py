"""Pins of the Fig. 5 programs: closed forms, exact rational brute force,
and the exact-rounded sum of the standard library."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import blas


@pytest.mark.parametrize("k", [0, 1, 5, 12, 20])
def test_asum_closed_form(k):
    # x_i = i/n, n = 2^k: every x_i and every partial sum is a dyadic
    # rational with < 53 bits, so the FP64 fold is exact: sum = (n-1)/2.
    n = 1 << k
    x = np.arange(n) / n
    assert blas.asum(x) == (n - 1) / 2
    # alternating signs: abs must undo them
    s = np.where(np.arange(n) % 2 == 1, -x, x)
    assert blas.asum(s) == (n - 1) / 2


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 1 << 16])
def test_dot_closed_forms(n):
    assert blas.dot(np.full(n, 0.5), np.full(n, 3.0)) == 1.5 * n
    i = np.arange(n, dtype=float)
    assert blas.dot(i, np.ones(n)) == n * (n - 1) / 2
    # sum i^2 = (n-1) n (2n-1) / 6
    assert blas.dot(i, i) == (n - 1) * n * (2 * n - 1) / 6


def test_gemv_closed_forms():
    M, N = 37, 53
    y = np.arange(M, dtype=float) - 10
    # A = 1, x = 1: y' = alpha*N + beta*y
    out = blas.gemv(np.ones((M, N)), np.ones(N), y, 2.0, 0.5)
    assert np.array_equal(out, 2.0 * N + 0.5 * y)
    # A_ij = i (row index), x_j = j: y'_i = alpha * i * N(N-1)/2 + beta*y_i;
    # a transposed A would give alpha * sum_j j*j instead.
    A = np.repeat(np.arange(M, dtype=float)[:, None], N, axis=1)
    x = np.arange(N, dtype=float)
    out = blas.gemv(A, x, y, 1.0, 0.5)
    assert np.array_equal(out, np.arange(M) * (N * (N - 1) / 2) + 0.5 * y)
    # A_ij = j: every row equals sum_j j * x_j
    A2 = np.repeat(np.arange(N, dtype=float)[None, :], M, axis=0)
    out = blas.gemv(A2, np.ones(N), y, 1.0, 0.0)
    assert np.array_equal(out, np.full(M, N * (N - 1) / 2))


def test_gemv_beta_zero_does_not_read_y():
    out = blas.gemv(np.ones((3, 4)), np.ones(4), np.full(3, np.nan), 1.0, 0.0)
    assert np.array_equal(out, np.full(3, 4.0))
    # beta != 0 reads y, and NaN propagates
    out = blas.gemv(np.ones((3, 4)), np.ones(4), np.full(3, np.nan), 1.0, 1.0)
    assert np.isnan(out).all()


def test_empty_inputs():
    assert blas.asum(np.zeros(0)) == 0.0
    assert blas.dot(np.zeros(0), np.zeros(0)) == 0.0
    assert blas.gemv(np.zeros((0, 3)), np.ones(3), np.zeros(0), 1.0, 1.0).size == 0
    out = blas.gemv(np.zeros((3, 0)), np.zeros(0), np.array([1.0, 2.0, 3.0]), 1.0, 0.5)
    assert out.tolist() == [0.5, 1.0, 1.5]


def _dyadic(rng, shape, bits=8):
    return rng.integers(-(1 << bits), 1 << bits, shape) / 16.0


@pytest.mark.parametrize("seed", range(8))
def test_brute_force_fractions(seed):
    """Tiny dyadic inputs: every FP64 operation is exact, so the oracle
    must equal the exact rational value computed with Fraction."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 17))
    x, y = _dyadic(rng, n), _dyadic(rng, n)
    assert blas.asum(x) == float(sum(abs(Fraction(v)) for v in x))
    assert blas.dot(x, y) == float(sum(Fraction(a) * Fraction(b) for a, b in zip(x, y)))
    a = 1.5
    assert blas.scal(a, x).tolist() == [float(Fraction(a) * Fraction(v)) for v in x]
    M = int(rng.integers(1, 6))
    A = _dyadic(rng, (M, n))
    yy = _dyadic(rng, M)
    out = blas.gemv(A, x, yy, 2.0, -0.5)
    exp = [float(Fraction(2) * sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(n))
                 + Fraction(-1, 2) * Fraction(yy[i])) for i in range(M)]
    assert out.tolist() == exp


@pytest.mark.parametrize("n", [10, 4097, 1 << 18])
def test_fold_within_fp64_bound_of_exact_sum(n):
    # math.fsum is the correctly rounded sum; a left fold in FP64 is within
    # (n-1) * 2^-53 * sum|t| of the exact value.
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    exact = math.fsum(np.abs(x))
    assert abs(blas.asum(x) - exact) <= n * 2 ** -53 * exact
    prods = x * y            # exact products would need 106 bits; bound both
    ex = math.fsum(prods)
    terms = math.fsum(np.abs(prods))
    assert abs(blas.dot(x, y) - ex) <= (n + 1) * 2 ** -53 * terms


def test_scal_fp32_product_is_correctly_rounded():
    # the FP64 product of two fp32 values is exact (48 significant bits), so
    # rounding it once to fp32 is the correctly rounded fp32 product.
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1000).astype(np.float32)
    out = blas.scal(1.5, x)
    for v, o in zip(x[:50], out[:50]):
        assert Fraction(float(v)) * Fraction(3, 2) == Fraction(float(o))


def test_tolerance_formula():
    u = 2.0 ** -24
    assert blas.tolerance(1 << 20, 10.0) == 4 * u * 20 * 10.0
    assert blas.tolerance(1, 3.0) == 4 * u * 1 * 3.0
    assert blas.tolerance(3, 1.0) == 4 * u * 2
    assert blas.tolerance(1000, 1.0) == 4 * u * 10


# ---------------------------------------------------------------------------
# user-function programs: nrm2, sum, axpy
# ---------------------------------------------------------------------------
def test_nrm2_closed_forms():
    assert blas.nrm2(np.array([3.0, 4.0])) == 5.0
    assert blas.nrm2(np.array([-3.0, 4.0])) == 5.0          # the square removes the sign
    for k in range(0, 12, 3):
        assert blas.nrm2(np.ones(4 ** k)) == 2.0 ** k        # sqrt(4^k)
    assert blas.nrm2(np.zeros(0)) == 0.0


def test_sum_closed_forms_and_signs():
    for n in (1, 7, 1 << 14):
        i = np.arange(n, dtype=float)
        assert blas.sum_(i) == n * (n - 1) / 2
        assert blas.sum_(-i) == -n * (n - 1) / 2              # no abs: signs stay


@pytest.mark.parametrize("seed", range(4))
def test_nrm2_sum_axpy_brute_force(seed):
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(1, 17))
    x, y = _dyadic(rng, n), _dyadic(rng, n)
    s2 = sum(Fraction(v) ** 2 for v in x)
    assert blas.nrm2(x) == math.sqrt(float(s2))             # S exact in FP64, sqrt rounded once
    assert blas.sum_(x) == float(sum(Fraction(v) for v in x))
    a = -0.75
    assert blas.axpy(a, x, y).tolist() == [float(Fraction(a) * Fraction(u) + Fraction(w))
                                           for u, w in zip(x, y)]


def test_axpy_fp32_rounds_twice():
    # fl(fl(a x) + y): the product is rounded before the add (no fused multiply-add)
    x = np.array([np.float32(1 + 2 ** -23)], np.float32)
    y = np.array([np.float32(-1.5)], np.float32)
    got = blas.axpy(1.5, x, y, mode="f32")[0]
    prod = np.float32(1.5 * (1 + 2 ** -23))                  # rounds 1.5 + 1.5*2^-23
    assert got == np.float32(prod + np.float32(-1.5))
    assert got != np.float32(1.5 * (1 + 2 ** -23) - 1.5)     # the fused value differs


def test_nrm2_tolerance_formula():
    u = 2.0 ** -24
    assert blas.nrm2_tolerance(1 << 20, 16.0) == (4 * 20 + 2) * u * 4.0


def test_gemv_t_closed_forms_and_transpose():
    M, N = 29, 41
    y = np.arange(N, dtype=float) - 5
    # A_ij = i (row index), x = 1: every column sums to M(M-1)/2
    A = np.repeat(np.arange(M, dtype=float)[:, None], N, axis=1)
    out = blas.gemv_t(A, np.ones(M), y, 2.0, 0.5)
    assert np.array_equal(out, 2.0 * M * (M - 1) / 2 + 0.5 * y)
    # A_ij = j: column j sums to j * sum(x); a non-transposed read would
    # give the row sums instead
    A2 = np.repeat(np.arange(N, dtype=float)[None, :], M, axis=0)
    x = np.arange(M, dtype=float)
    out = blas.gemv_t(A2, x, y, 1.0, 0.0)
    assert np.array_equal(out, np.arange(N) * (M * (M - 1) / 2))
    # the reorder-stride view is the transpose
    from oracle.patterns import evaluate
    B = np.arange(M * N, dtype=float).reshape(M, N)
    assert np.array_equal(evaluate(blas.transpose_expr(M, N), B), B.T)


@pytest.mark.parametrize("seed", range(3))
def test_gemv_t_brute_force(seed):
    rng = np.random.default_rng(90 + seed)
    M, N = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    A, x, y = _dyadic(rng, (M, N)), _dyadic(rng, M), _dyadic(rng, N)
    out = blas.gemv_t(A, x, y, -1.5, 0.25)
    exp = [float(Fraction(-3, 2) * sum(Fraction(A[i, j]) * Fraction(x[i]) for i in range(M))
                 + Fraction(1, 4) * Fraction(y[j])) for j in range(N)]
    assert out.tolist() == exp
    assert blas.gemv_t(np.zeros((0, N)), np.zeros(0), y, 1.0, 0.5).tolist() == (0.5 * y).tolist()


def test_exact_sums_are_correctly_rounded():
    # a left fold loses the 1 entirely; the exact sums keep it
    x = np.array([2.0 ** 60, 1.0, -(2.0 ** 60)])
    assert blas.dot_exact(x, np.ones(3)) == 1.0
    assert blas.asum_exact(np.array([2.0 ** 52, 0.5, -(2.0 ** 52)])) == 2.0 ** 53   # ties to even
    # a left fold rounds 1 + 2^-53 back to 1 twice; the exact sum is 1 + 2^-52
    assert blas.asum_exact(np.array([1.0, -(2.0 ** -53), 2.0 ** -53])) == 1 + 2.0 ** -52
    assert blas.asum(np.array([1.0, -(2.0 ** -53), 2.0 ** -53])) == 1.0
    # fp32 products are exact in FP64: (1 + 2^-23)^2 = 1 + 2^-22 + 2^-46
    a = np.array([np.float32(1 + 2 ** -23)], np.float32)
    assert blas.dot_exact(a, a) == 1 + 2 ** -22 + 2 ** -46
    rng = np.random.default_rng(4)
    p = rng.integers(-(1 << 20), 1 << 20, 5000).astype(float)
    q = rng.integers(-(1 << 20), 1 << 20, 5000).astype(float)
    assert blas.dot_exact(p, q) == float(int(np.sum(p.astype(object) * q.astype(object))))


def test_compensated_tolerance_formula():
    u = 2.0 ** -24
    assert blas.compensated_tolerance(-3.0, 100.0, 10) == 2 * u * 3 + 2 * (10 * u) ** 2 * 100
