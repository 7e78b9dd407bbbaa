"""The rewrite rules (Fig. 3, Fig. 4) preserve values; the printed
derivation of Fig. 8 and the expressions of Fig. 2b and Fig. 9 evaluate to
the programs they were derived from."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import blas
from oracle import lowlevel as ll
from oracle import rules as R
from oracle.patterns import (ArrT, AsVector, C, Id, Iterate, Join, Map, MapSeq,
                             PartRed, PatternTypeError, Reduce, ReduceSeq,
                             Reorder, Split, TupT, Vect, Zip, abs_, add,
                             evaluate, infer, mul3, mult, mult_by)


def test_fig8_derivation_by_rules():
    """Apply the rules named above each equality of Fig. 8 and land on each
    printed equation in turn; every equation evaluates to asum."""
    n = 64
    eqs = ll.fig8_equations(n)
    t = ArrT((4096,))
    e = eqs[0]
    e = R.rewrite(e, (0,), "reduction")                       # 3d
    e = R.rewrite(e, (1,), "partred_split", n=n)              # 3d
    assert e == eqs[1]
    e = R.rewrite(e, (4,), "split_join", n=n)                 # 3c
    assert e == eqs[2]
    e = R.rewrite(e, (), "simplify_split_join", t=t, at=3)    # 3e
    e = R.rewrite(e, (), "drop_id", at=2)
    assert e == eqs[3]
    e = R.rewrite(e, (), "fuse_maps", at=2)                   # 3f
    assert e == eqs[4]
    e = R.rewrite(e, (2, "f", 1), "lower_map", kind="map-seq")  # 4a
    assert e == eqs[5]
    e = R.rewrite(e, (2, "f", 0), "partred_to_reduce")        # 3d
    e = R.rewrite(e, (2, "f", 0), "lower_reduce")             # 4b
    assert e == eqs[6]
    e = R.rewrite(e, (2, "f"), "fuse_reduce_seq", at=0)       # 3f
    assert e == eqs[7]
    x = np.random.default_rng(0).integers(-1000, 1000, 4096).astype(float)
    ref = float(np.abs(x).sum())
    for q in eqs:
        assert evaluate(q, x)[0] == ref


def test_simplification_needs_matching_sizes():
    t = ArrT((64,))
    e = C(Split(8), Join(), Split(4))          # join of [16][4], then split-8
    with pytest.raises(R.NotApplicable):
        R.rewrite(e, (), "simplify_split_join", t=t, at=0)


def test_fig9_types_and_values():
    g = read_golden("fig9_parameters.txt")
    n = 1 << 20
    t = ArrT((n,))
    for e in (ll.fig9a_nvidia(), ll.fig9b_amd(), ll.fig9c_intel()):
        assert infer(e, t).dims == (1,)
    # (a): the workgroup chunk splits into threads x thread-chunk
    a_wg, a_tc = int(g["a_workgroup_chunk"]), int(g["a_thread_chunk"])
    assert a_wg // a_tc == int(g["a_threads"]) == 2 ** int(g["a_iterations"])
    b_v = int(g["b_workgroup_chunk"]) // int(g["b_vector"])
    assert b_v // 2 == int(g["b_threads"]) == 2 ** int(g["b_iterations"])
    assert int(g["c_workgroup_chunk"]) // int(g["c_vector"]) // 8192 == int(g["c_threads"])
    x = np.random.default_rng(1).integers(-50, 50, n).astype(float)
    ref = float(np.abs(x).sum())
    for e in (ll.fig9a_nvidia(), ll.fig9b_amd(), ll.fig9c_intel()):
        assert evaluate(e, x)[0] == ref


def _replace_first(e, old, new):
    """Replace the first node equal to ``old``."""
    for p in R.positions(e):
        node = e
        for s in p:
            node = R._child(node, s)
        if node == old:
            return R._replace(e, p, new)
    raise AssertionError("not found")


@pytest.mark.parametrize("bad", [
    (Split(2048), Split(2047)),
    (Iterate(7, C(Join(), ll.MapLocal(ReduceSeq(add, 0)), Split(2))),
     Iterate(8, C(Join(), ll.MapLocal(ReduceSeq(add, 0)), Split(2)))),
    (Split(262144), Split(262143)),
])
def test_fig9a_perturbed_parameters_rejected(bad):
    e = _replace_first(ll.fig9a_nvidia(), *bad)
    with pytest.raises(PatternTypeError):
        infer(e, ArrT((1 << 20,)))


def test_fig9bc_perturbed_parameters_rejected():
    b = ll.fig9b_amd()
    it8 = [p for p in R.positions(b) if isinstance(_node(b, p), Iterate)][0]
    bad = R._replace(b, it8, Iterate(9, _node(b, it8).f))
    with pytest.raises(PatternTypeError):
        infer(bad, ArrT((1 << 20,)))
    c = _replace_first(ll.fig9c_intel(), Split(8192), Split(8191))
    with pytest.raises(PatternTypeError):
        infer(c, ArrT((1 << 20,)))
    c = _replace_first(ll.fig9c_intel(), AsVector(4), AsVector(3))
    with pytest.raises(PatternTypeError):
        infer(c, ArrT((1 << 20,)))


def _node(e, p):
    for s in p:
        e = R._child(e, s)
    return e


def test_fig2b_vector_scal():
    x = np.arange(4096, dtype=np.int64)
    out = evaluate(ll.fig2b_vector_scal(), x, mode="int")
    assert np.array_equal(out, 3 * x)
    assert np.array_equal(out, evaluate(Map(mul3), x, mode="int"))
    with pytest.raises(PatternTypeError):
        evaluate(ll.fig2b_vector_scal(), np.arange(1000, dtype=np.int64), mode="int")


def test_vectorization_rule_applies_once():
    e = Map(abs_)
    v = R.rewrite(e, (), "vectorize", n=4)
    inner = v.fs[1]
    assert isinstance(inner.f, Vect)
    with pytest.raises(R.NotApplicable):
        R.rewrite(v, (1,), "vectorize", n=4)


# ---------------------------------------------------------------------------
# random derivations
# ---------------------------------------------------------------------------
PROGRAMS = {
    "asum": (blas.asum_expr(), lambda rng, n: rng.integers(-99, 99, n).astype(float)),
    "scal": (blas.scal_expr(3), lambda rng, n: rng.integers(-99, 99, n).astype(float)),
    "dot": (blas.dot_expr(), lambda rng, n: (rng.integers(-99, 99, n).astype(float),
                                            rng.integers(-9, 9, n).astype(float))),
}


def _candidates(e, t, rng):
    """(path, rule, params) triples that apply to ``e``."""
    out = []
    for p in R.positions(e):
        node = _node(e, p)
        for name in R.NODE_RULES:
            params = {}
            if name in ("split_join", "partred_split", "vectorize"):
                params = {"n": int(rng.choice([2, 4]))}
            elif name == "partred_iterate":
                params = {"n": 1}
            elif name == "iterate_decomposition":
                params = {"m": int(rng.integers(0, 3))}
            elif name == "lower_map":
                params = {"kind": str(rng.choice(["map-workgroup", "map-local", "map-seq"]))}
            elif name == "lower_reorder":
                params = {"n": int(rng.choice([2, 4]))} if rng.random() < 0.5 else {}
            try:
                new = R.rewrite(e, p, name, t=t, **params)
            except (R.NotApplicable, PatternTypeError, AttributeError, TypeError):
                continue
            out.append((name, new))
        if isinstance(node, type(C(Id(), Id()))):
            for i in range(len(node.fs) - 1):
                for name in R.PAIR_RULES:
                    try:
                        new = R.rewrite(e, p, name, t=t, at=i)
                    except (R.NotApplicable, PatternTypeError, AttributeError, TypeError):
                        continue
                    out.append((name, new))
    return [c for c in out if R.well_typed(c[1], t)]


EXPANDING = {"reduction", "partred_split", "split_join", "partred_iterate", "vectorize",
             "partred_reorder", "iterate_decomposition", "reorder_commutativity"}


def _pick(cands, rng, step):
    w = np.array([4.0 if (n in EXPANDING and step < 8) else 1.0 for n, _ in cands])
    return cands[int(rng.choice(len(cands), p=w / w.sum()))][1]


@pytest.mark.parametrize("prog", sorted(PROGRAMS))
@pytest.mark.parametrize("seed", range(10))
def test_random_derivations_preserve_value(prog, seed):
    rng = np.random.default_rng(100 + seed)
    e, gen = PROGRAMS[prog]
    n = 64
    x = gen(rng, n)
    t = TupT((ArrT((n,)), ArrT((n,)))) if isinstance(x, tuple) else ArrT((n,))
    ref = evaluate(e, x)
    for step in range(14):
        cands = _candidates(e, t, rng)
        if not cands:
            break
        e = _pick(cands, rng, step)
        got = evaluate(e, x)
        assert np.array_equal(got.reshape(-1), np.asarray(ref).reshape(-1)), repr(e)


def test_reorder_lowering_and_commutativity():
    x = np.arange(16.0) - 8
    e = C(Map(abs_), Reorder())
    e2 = R.rewrite(e, (), "reorder_commutativity", at=0)
    assert isinstance(e2.fs[0], Reorder)
    # the strided lowering permutes a map's output -- the value is a
    # permutation, and reduce(+) over it is unchanged
    e3 = R.rewrite(e, (1,), "lower_reorder", s=4)
    out = evaluate(e3, x)
    assert sorted(out.tolist()) == sorted(np.abs(x).tolist())
    red = C(Reduce(add, 0), e3)
    assert evaluate(red, x)[0] == np.abs(x).sum()


# ---------------------------------------------------------------------------
# kernel-variant expressions compute the Fig. 5 programs
# ---------------------------------------------------------------------------
VARIANTS = [
    # tile, vw, threads, grid, stride, cluster, ft
    (256, 1, 32, 5, True, 1, 32),
    (1024, 4, 256, 3, True, 1, 256),
    (1024, 4, 256, 3, False, 1, 256),
    (2048, 8, 256, 4, True, 2, 256),
    (4096, 8, 256, 8, True, 4, 256),
]


@pytest.mark.parametrize("n", [1, 255, 4096, 20000])
@pytest.mark.parametrize("v", VARIANTS)
def test_reduce_variant_expressions_are_exact_on_integers(n, v):
    tile, vw, th, g, st, cl, ft = v
    rng = np.random.default_rng(n)
    x = rng.integers(-500, 500, n).astype(float)
    y = rng.integers(-9, 9, n).astype(float)
    e, L = ll.reduce_variant("asum", n, tile, vw, th, g, st, cl, ft)
    xp = np.concatenate([x, np.zeros(L - n)])
    assert evaluate(e, xp)[0] == np.abs(x).sum()
    e, L = ll.reduce_variant("dot", n, tile, vw, th, g, st, cl, ft)
    yp = np.concatenate([y, np.zeros(L - n)])
    assert evaluate(e, (xp, yp))[0] == x @ y


def test_padding_does_not_change_the_definition():
    # Reading of a ragged tail: padding with the neutral element 0 leaves
    # asum and dot unchanged (abs(0) = 0, 0 * y = 0, acc + 0 = acc).
    x = np.arange(1, 11, dtype=float)
    assert blas.asum(np.concatenate([x, np.zeros(6)])) == blas.asum(x)
    assert blas.dot(np.concatenate([x, np.zeros(6)]),
                    np.concatenate([x, np.full(6, 7.0)])) == blas.dot(x, x)


@pytest.mark.parametrize("N,vw", [(1, 1), (33, 4), (256, 8), (1000, 4)])
def test_gemv_variant_expression_exact(N, vw):
    rng = np.random.default_rng(N)
    M = 6
    A = rng.integers(-9, 9, (M, N)).astype(float)
    x = rng.integers(-9, 9, N).astype(float)
    z = evaluate(ll.gemv_z_variant(M, N, 2.0, vw, 32, 2), A, env={"x": x})
    assert np.array_equal(z, 2.0 * (A @ x))


@pytest.mark.parametrize("n,item,tile,vw", [(0, 1024, 1024, 1), (1, 2048, 1024, 4),
                                            (5000, 2048, 1024, 4), (70001, 8192, 4096, 8)])
def test_batch_expression_exact_on_integers(n, item, tile, vw):
    rng = np.random.default_rng(n + 1)
    x = rng.integers(-500, 500, n).astype(float)
    y = rng.integers(-9, 9, n).astype(float)
    # cast32=False: the FP64 combine before the final rounding to fp32
    e, Lp = ll.batch_reduce("asum", n, item, tile, vw, cast32=False)
    xp = np.concatenate([x, np.zeros(Lp - n)])
    assert evaluate(e, xp)[0] == np.abs(x).sum()
    e, Lp = ll.batch_reduce("dot", n, item, tile, vw, cast32=False)
    yp = np.concatenate([y, np.zeros(Lp - n)])
    assert evaluate(e, (xp, yp))[0] == x @ y


@pytest.mark.parametrize("op", ["nrm2", "sum"])
@pytest.mark.parametrize("n", [1, 5000, 20000])
def test_user_function_variant_expressions_exact(op, n):
    rng = np.random.default_rng(n + 7)
    x = rng.integers(-50, 50, n).astype(float)
    e, Lp = ll.reduce_variant(op, n, 1024, 4, 256, 3, True, 1, 256, cast32=False)
    xp = np.concatenate([x, np.zeros(Lp - n)])
    got = evaluate(e, xp)[0]
    if op == "nrm2":
        assert got == np.sqrt(float((x * x).sum()))
    else:
        assert got == x.sum()


@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("M,N,B", [(1, 1, 1), (37, 20, 8), (64, 33, 64), (100, 7, 3),
                                   (200, 5, 2)])
def test_gemv_t_variant_expression_exact(M, N, B, passes):
    # integer inputs: every operation is exact, so any combine order must
    # give the exact A^T x (a dropped block, lane or tree level would not)
    rng = np.random.default_rng(M * N)
    A = rng.integers(-9, 9, (M, N)).astype(float)
    x = rng.integers(-9, 9, M).astype(float)
    RB = -(-M // B)
    z = evaluate(ll.gemv_t_z_variant(M, N, 2.0, B, RB, passes), A, env={"x": x})
    assert np.array_equal(z, 2.0 * (A.T @ x))


@pytest.mark.parametrize("M,N,vw,threads,L,S", [(3, 1000, 4, 64, 256, 4), (2, 5, 1, 32, 32, 1),
                                                 (4, 700, 2, 32, 64, 11), (1, 4200, 1, 64, 64, 66)])
def test_gemv_split_variant_expression_exact(M, N, vw, threads, L, S):
    # integer inputs: exact in any order, so the segments, lanes and trees
    # must together cover every product exactly once
    rng = np.random.default_rng(N)
    A = rng.integers(-9, 9, (M, N)).astype(float)
    x = rng.integers(-9, 9, N).astype(float)
    z = evaluate(ll.gemv_split_z_variant(M, N, 2.0, vw, threads, L, S), A, env={"x": x})
    assert np.array_equal(z, 2.0 * (A @ x))


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("M,N,B", [(1, 1, 1), (37, 20, 8), (64, 33, 4), (100, 7, 3)])
def test_gemv_t_cluster_expression_exact(M, N, B, cluster):
    # the cluster form pads the block count to whole clusters (blocks of
    # zero rows); on integer inputs it must still give exactly A^T x -- a
    # dropped cluster, block or padding mistake would not
    rng = np.random.default_rng(M * N + cluster)
    A = rng.integers(-9, 9, (M, N)).astype(float)
    x = rng.integers(-9, 9, M).astype(float)
    RB = -(-M // B)
    RB = -(-RB // cluster) * cluster
    z = evaluate(ll.gemv_t_z_variant(M, N, 2.0, B, RB, 1, cluster), A, env={"x": x})
    assert np.array_equal(z, 2.0 * (A.T @ x))
