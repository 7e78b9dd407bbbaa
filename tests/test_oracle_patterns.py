"""Pins of the pattern interpreter against the definitions of Sec. 3
(Table 1, Table 2) -- independent of the interpreter's own code paths."""
import numpy as np
import pytest

from conftest import read_golden
from oracle.patterns import (AsScalar, AsVector, C, Id, Iterate, Join, Map,
                             MapLocal, MapSeq, MapWorkgroup, PadTo,
                             PatternTypeError, Reduce, ReduceSeq, Reorder,
                             ReorderStride, Split, ToLocal, Vect, Zip, abs_,
                             absAndPlus, add, add64, evaluate, fold, mult,
                             mult_by, to_f32)


def ints(s):
    return [int(t) for t in s.split()]


def test_reorder_stride_matches_worked_example():
    g = read_golden("reorder_stride.txt")
    out = evaluate(ReorderStride(s=int(g["s"])), np.array(ints(g["input"]), float))
    assert out.tolist() == ints(g["output"])
    out = evaluate(ReorderStride(s=int(g["s12"])), np.array(ints(g["input12"]), float))
    assert out.tolist() == ints(g["output12"])
    # the n form: s = len / n
    out = evaluate(ReorderStride(n=4), np.arange(8.0))
    assert out.tolist() == ints(g["output"])


def test_reorder_stride_is_a_transpose():
    # reorder-stride^s on s*n elements reads the s x n row-major matrix by
    # columns, i.e. it is the transpose of an n x s matrix stored row-major.
    s, n = 6, 5
    x = np.arange(s * n, dtype=float)
    out = evaluate(ReorderStride(s=s), x)
    assert np.array_equal(out, x.reshape(n, s).T.reshape(-1))


def test_split_join_shapes_and_errors():
    x = np.arange(12.0)
    assert evaluate(Split(4), x).shape == (3, 4)
    assert evaluate(Split(4), x)[1].tolist() == [4, 5, 6, 7]
    assert np.array_equal(evaluate(C(Join(), Split(3)), x), x)
    with pytest.raises(PatternTypeError):
        evaluate(Split(5), x)          # the size must divide (the type carries it)
    with pytest.raises(PatternTypeError):
        evaluate(Join(), x)            # join needs two dimensions


def test_iterate_definition():
    # f^0 = id and f^(n+1) = f^n . f  (Sec. 3.1)
    f = C(Join(), Map(Reduce(add, 0)), Split(2))
    x = np.arange(16.0)
    assert np.array_equal(evaluate(Iterate(0, f), x), x)
    step1 = evaluate(f, x)
    assert step1.tolist() == [1, 5, 9, 13, 17, 21, 25, 29]
    assert evaluate(Iterate(4, f), x).tolist() == [120.0]
    with pytest.raises(PatternTypeError):
        evaluate(Iterate(5, f), x)     # 1 element cannot be split in 2


def test_reduce_is_left_fold_from_z():
    # reduce(f, z): acc = z; acc = f(acc, x_i) in order.  With a
    # non-commutative, non-associative check function (mult then add with
    # a marker) the order is visible; here: z = 5, add -> 5 + sum.
    x = np.array([1.0, 2.0, 3.0])
    assert evaluate(Reduce(add, 5), x).tolist() == [11.0]
    assert evaluate(Reduce(mult, 2), x).tolist() == [12.0]
    # fold order: (((z + x0) + x1) + x2) in fp32 differs from the other
    # association for these values.
    big, small = np.float32(2 ** 24), np.float32(1.0)
    v = np.array([big, small, small], np.float32)
    left = evaluate(ReduceSeq(add, 0), v, mode="f32")[0]
    assert left == np.float32(2 ** 24)     # 2^24 + 1 rounds back to 2^24 twice
    v2 = np.array([small, small, big], np.float32)
    assert evaluate(ReduceSeq(add, 0), v2, mode="f32")[0] == np.float32(2 ** 24 + 2)


@pytest.mark.parametrize("mode,dt", [("f64", np.float64), ("f32", np.float32)])
def test_fused_fold_matches_python_loop(mode, dt):
    """The vectorised fold must perform exactly the loop's operations in
    the loop's order (checked against an explicit scalar loop)."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal(3001).astype(np.float32)
    y = rng.standard_normal(3001).astype(np.float32)
    acc = dt(0)
    for a in x.astype(dt):
        acc = dt(acc + (-a if a < 0 else a))
    got = evaluate(ReduceSeq(absAndPlus, 0), x, mode=mode)[0]
    assert got == acc
    acc = dt(0)
    for a, b in zip(x.astype(dt), y.astype(dt)):
        acc = dt(acc + dt(a * b))
    got = evaluate(C(ReduceSeq(fold(add, mult), 0), Zip()), (x, y), mode=mode)[0]
    assert got == acc


def test_fold_longer_than_chunk_keeps_order(monkeypatch):
    import oracle.patterns as P
    monkeypatch.setattr(P, "FOLD_CHUNK", 7)
    x = np.random.default_rng(1).standard_normal(100).astype(np.float32)
    acc = np.float32(0)
    for a in x:
        acc = np.float32(acc + a)
    assert evaluate(ReduceSeq(add, 0), x, mode="f32")[0] == acc


def test_abs_follows_fig5_definition():
    # abs(x) = if (x < 0) -x else x : -0.0 stays -0.0, NaN stays NaN
    out = evaluate(Map(abs_), np.array([-2.0, 3.0, -0.0, np.nan]))
    assert out[0] == 2.0 and out[1] == 3.0
    assert np.signbit(out[2]) and np.isnan(out[3])


def test_vectors():
    x = np.arange(8.0)
    v = evaluate(AsVector(4), x)
    assert v.shape == (2, 4) and v[1].tolist() == [4, 5, 6, 7]
    assert np.array_equal(evaluate(C(AsScalar(), AsVector(4)), x), x)
    with pytest.raises(PatternTypeError):
        evaluate(AsVector(3), x)
    with pytest.raises(PatternTypeError):
        evaluate(Map(abs_), np.zeros((2, 2)))       # user function over arrays
    with pytest.raises(PatternTypeError):
        evaluate(C(Map(abs_), AsVector(4)), x)      # scalar function over vectors
    out = evaluate(C(AsScalar(), Map(Vect(4, abs_)), AsVector(4)), -x)
    assert np.array_equal(out, x)
    # a vectorised fold accumulates lane by lane
    acc = evaluate(C(ReduceSeq(Vect(4, absAndPlus), 0), AsVector(4)), -x)
    assert acc.tolist() == [[4.0, 6.0, 8.0, 10.0]]


def test_zip_requires_equal_lengths():
    with pytest.raises(PatternTypeError):
        evaluate(C(Map(mult), Zip()), (np.ones(3), np.ones(4)))
    out = evaluate(C(Map(mult), Zip()), (np.arange(3.0), np.arange(3.0)))
    assert out.tolist() == [0, 1, 4]


def test_thread_hierarchy_is_checked():
    x = np.arange(16.0)
    with pytest.raises(PatternTypeError):   # map-local outside map-workgroup
        evaluate(C(Join(), MapLocal(Map(abs_)), Split(4)), x)
    with pytest.raises(PatternTypeError):   # map-workgroup inside map-workgroup
        evaluate(C(Join(), MapWorkgroup(C(Join(), MapWorkgroup(Map(abs_)), Split(2))), Split(4)), x)
    with pytest.raises(PatternTypeError):   # map-local inside map-local
        evaluate(C(Join(), MapWorkgroup(C(Join(), MapLocal(C(Join(), MapLocal(Map(abs_)), Split(2))),
                                            Split(2))), Split(4)), x)
    with pytest.raises(PatternTypeError):   # parallel map inside a sequential one
        evaluate(C(Join(), MapWorkgroup(C(Join(), MapSeq(MapLocal(abs_)), Split(2))), Split(4)), x)
    ok = C(Join(), MapWorkgroup(C(Join(), ToLocal(MapLocal(MapSeq(abs_))), Split(2))), Split(4))
    assert np.array_equal(evaluate(ok, -x), x)


def test_reorder_is_identity_and_pad():
    x = np.arange(5.0)
    assert np.array_equal(evaluate(Reorder(), x), x)
    assert evaluate(PadTo(8), x).tolist() == [0, 1, 2, 3, 4, 0, 0, 0]


def test_fp32_mode_rounds_each_operation():
    # 1 + 2^-24 is not representable: fp32 add rounds it back to 1 (ties to even)
    x = np.array([1.0, 2 ** -24, 2 ** -24], np.float32)
    assert evaluate(ReduceSeq(add, 0), x, mode="f32")[0] == np.float32(1.0)
    # add64 keeps it: 1 + 2^-23 exactly, then to_f32 rounds to 1 + 2^-23
    r = evaluate(C(Map(to_f32), ReduceSeq(add64, 0)), x, mode="f32")[0]
    assert r == np.float32(1.0 + 2 ** -23)
    # 1.5 * x: the product of two fp32 values rounded once
    v = np.array([np.float32(1 + 2 ** -23)], np.float32)
    got = evaluate(Map(mult_by(1.5)), v, mode="f32")[0]
    exact = 1.5 * (1 + 2 ** -23)          # = 1.5 + 1.5*2^-23, needs 25 bits
    assert got == np.float32(exact) and got.dtype == np.float32
    with pytest.raises(ValueError):
        evaluate(Map(abs_), np.array([0.1]), mode="f32")   # 0.1 is not an fp32 value


# ---------------------------------------------------------------------------
# the compensated reduce-seq (Neumaier's summation) used for the lane folds
# ---------------------------------------------------------------------------
def test_reduce_seq_comp_exact_on_integers():
    from oracle.patterns import ReduceSeqComp
    rng = np.random.default_rng(3)
    x = rng.integers(-1000, 1000, 777)
    assert evaluate(ReduceSeqComp(), x, mode="int")[0] == int(x.sum())
    assert evaluate(ReduceSeqComp(), x.astype(float))[0] == float(x.sum())


def test_reduce_seq_comp_recovers_what_a_plain_fold_loses():
    # 1 followed by 100 terms of 2^-24: each plain fp32 add is a tie that
    # rounds back to 1 (round to even), so the plain left fold returns 1;
    # the exact sum 1 + 100 * 2^-24 = 1 + 50 * 2^-23 is an fp32 number, and
    # the compensated fold returns it exactly
    from oracle.patterns import ReduceSeqComp
    x = np.concatenate([[1.0], np.full(100, 2.0 ** -24)])
    assert evaluate(ReduceSeq(add, 0), x, mode="f32")[0] == np.float32(1.0)
    assert evaluate(ReduceSeqComp(), x, mode="f32")[0] == np.float32(1.0 + 100 * 2.0 ** -24)
    # the smaller operand first (the other branch of the correction)
    y = np.concatenate([np.full(100, 2.0 ** -24), [1.0], np.full(100, -(2.0 ** -24))])
    assert evaluate(ReduceSeqComp(), y, mode="f32")[0] == np.float32(1.0)


def test_reduce_seq_comp_keeps_inf_and_nan():
    from oracle.patterns import ReduceSeqComp
    assert evaluate(ReduceSeqComp(), np.array([1.0, np.inf, 2.0]), mode="f32")[0] == np.inf
    assert evaluate(ReduceSeqComp(), np.array([1.0, -np.inf, 2.0]), mode="f32")[0] == -np.inf
    assert np.isnan(evaluate(ReduceSeqComp(), np.array([1.0, np.nan, 2.0]), mode="f32")[0])


@pytest.mark.parametrize("seed", range(5))
def test_reduce_seq_comp_within_two_units_of_the_exact_sum(seed):
    # Neumaier's bound: |s_comp - S| <= 2u|S| + 2 m^2 u^2 sum|x_i| (u = 2^-24)
    import math
    from oracle.patterns import ReduceSeqComp
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(3000) * np.exp(rng.uniform(-8, 8, 3000))).astype(np.float32)
    exact = math.fsum(float(v) for v in x)
    got = float(evaluate(ReduceSeqComp(), x.astype(np.float64), mode="f32")[0])
    u = 2.0 ** -24
    bound = 2 * u * abs(exact) + 2 * (3000 * u) ** 2 * float(np.abs(x.astype(np.float64)).sum())
    assert abs(got - exact) <= bound
    # a plain fp32 left fold of the same terms is typically far worse
    plain = float(evaluate(ReduceSeq(add, 0), x.astype(np.float64), mode="f32")[0])
    assert abs(got - exact) <= abs(plain - exact)


def test_reduce_seq_comp_lanes():
    # vect^4(add): four independent compensated folds, lane by lane
    from oracle.patterns import ReduceSeqComp, Vect
    x = np.zeros((101, 4))
    x[0] = [1.0, 2.0, 4.0, 8.0]
    x[1:] = 2.0 ** -24
    got = evaluate(C(ReduceSeqComp(Vect(4, add)), AsVector(4)), x.reshape(-1), mode="f32")
    assert got.shape[-1] == 4
    # each lane returns the fp32 rounding of its exact sum
    for k, base in enumerate([1.0, 2.0, 4.0, 8.0]):
        assert got[0, k] == np.float32(base + 100 * 2.0 ** -24)
