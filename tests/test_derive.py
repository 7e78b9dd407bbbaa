"""Rule-driven enumeration: every derivation the enumerator produces is
checked against the oracle's interpreter (the derived low-level expression
must compute the high-level program exactly on integer inputs), the
parameters read off each expression match the choices that produced it, the
library variants the derivations reach are the ones whose parameters the
rules can express, and the emitted instantiation list is current."""
import os

import numpy as np
import pytest

from oracle import patterns as P
from paper_1502_02389_gb300 import derive as D

_FN = {"add": P.add, "abs": P.abs_, "mult": P.mult, "square": P.square, "id": P.id_}


def fn(f):
    if f.name == "fold":
        return P.fold(fn(f.args[0]), fn(f.args[1]))
    if f.name == "vect":
        return P.Vect(f.args[0], fn(f.args[1]))
    if f.name == "mult_by":
        return P.mult_by(3.0)
    return _FN[f.name]


def to_oracle(e):
    """The enumerator's expression as an oracle expression."""
    if isinstance(e, D.C):
        return P.C(*[to_oracle(f) for f in e.fs])
    if isinstance(e, D.Fn):
        return fn(e)
    if isinstance(e, D.Map):
        return P.Map(fn(e.f) if isinstance(e.f, D.Fn) else to_oracle(e.f), e.kind)
    if isinstance(e, D.Reduce):
        return P.Reduce(fn(e.f), e.z, e.kind)
    if isinstance(e, D.Split):
        return P.Split(e.n)
    if isinstance(e, D.Join):
        return P.Join()
    if isinstance(e, D.ReorderStride):
        return P.ReorderStride(s=e.s) if e.s else P.ReorderStride(n=e.n)
    if isinstance(e, D.AsVector):
        return P.AsVector(e.n)
    if isinstance(e, D.AsScalar):
        return P.AsScalar()
    if isinstance(e, D.Iterate):
        return P.Iterate(e.k, to_oracle(e.f))
    if isinstance(e, D.ToLocal):
        if e.f == D.Map("map-local", D.ID):        # the staging copy (also of zipped pairs)
            return P.ToLocal(P.Id())
        return P.ToLocal(to_oracle(e.f))
    if isinstance(e, D.Pad):
        return P.PadTo(e.n)
    if isinstance(e, D.ZipWith):
        return P.ZipWith(e.name)
    raise TypeError(e)


def high_level(op):
    return {"asum": P.C(P.Reduce(P.add, 0), P.Map(P.abs_)),
            "sum": P.Reduce(P.add, 0),
            "dot": P.C(P.Reduce(P.add, 0), P.Map(P.mult), P.Zip()),
            "scal": P.Map(P.mult_by(3.0))}[op]


def inputs(op, n, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(-50, 50, n).astype(float)
    if op == "dot":
        return (x, rng.integers(-50, 50, n).astype(float))
    return x


@pytest.mark.parametrize("op", ["asum", "dot", "sum"])
def test_every_reduction_derivation_computes_the_program(op):
    ders = list(D.derive(op))
    assert len(ders) > 200
    rng = np.random.default_rng(1)
    for d in [ders[i] for i in rng.choice(len(ders), 60, replace=False)]:
        tile = d.choice["tile"]
        x = inputs(op, 2 * tile, tile)
        e = to_oracle(d.expr)
        if op == "dot":
            e = P.C(e, P.Zip())
        got = P.evaluate(e, x)
        want = P.evaluate(high_level(op), x)
        assert np.array_equal(np.asarray(got), np.asarray(want)), (d.choice, d.expr)


def test_every_map_derivation_computes_the_program():
    for d in D.derive("scal"):
        x = inputs("scal", 2 * d.choice["tile"], 5)
        got = P.evaluate(to_oracle(d.expr), x)
        assert np.array_equal(np.asarray(got), 3.0 * x), d.choice


GEMV_Z = P.C(P.Join(), P.Map(P.C(P.Map(P.mult_by(3.0)), P.Reduce(P.add, 0), P.Map(P.mult),
                                 P.ZipWith("x"))))


def test_every_gemv_derivation_computes_the_program():
    """Fig. 5's gemv z = join . map(scal(a) . dot(x)) over the rows of A: each
    derivation -- a warp per row (rows per work-group, vector width, strided
    or contiguous work-item order, staged or not) or each row split over
    work-groups (work-items, vector width, order, segment length) --
    evaluates to the program exactly on integer inputs."""
    ders = list(D.derive("gemv"))
    warp = [d for d in ders if not d.choice.get("split")]
    split = [d for d in ders if d.choice.get("split")]
    assert len(warp) == len(D.GEMV_ROWS) * len(D.WIDTHS) * 2 * 2 and len(split) > 50
    rng = np.random.default_rng(4)
    for d in warp + [split[i] for i in rng.choice(len(split), 20, replace=False)]:
        M, N = 2 * d.choice.get("rows", 1), d.choice["n"]
        A = rng.integers(-20, 20, (M, N)).astype(float)
        x = rng.integers(-20, 20, N).astype(float)
        got = P.evaluate(to_oracle(d.expr), A, env={"x": x})
        want = P.evaluate(GEMV_Z, A, env={"x": x})
        assert np.array_equal(np.asarray(got), np.asarray(want)), d.choice
        assert np.array_equal(np.asarray(want), 3.0 * (A @ x))


def test_gemv_parameters_read_back_the_choices():
    for d in D.derive("gemv"):
        p = D.parameters(d.expr)
        c = d.choice
        if c.get("split"):
            assert p == dict(kind="gemv_split", threads=c["threads"], vw=c["vw"],
                             strided=c["strided"]), (c, p)
        else:
            assert p == dict(kind="gemv", rows=c["rows"], vw=c["vw"], lanes=32,
                             strided=c["strided"], staged=c["staged"]), (c, p)
    # a tree that is not the 32-lane halving tree has no template
    d = D.derive_gemv(8, 4, True)
    row = list(D.parts(d.expr.fs[2].f.f))
    row[1] = D.Iterate(4, row[1].f)
    bad = D.comp(*(list(d.expr.fs[:2]) + [D.Map("map-workgroup", D.Map("map", D.comp(*row)))]
                   + [d.expr.fs[3]]))
    assert D.parameters(bad) is None


def test_parameters_read_back_the_choices():
    seen_rejected = 0
    for op in ("asum", "dot", "scal"):
        for d in D.derive(op):
            p = D.parameters(d.expr)
            c = d.choice
            if op != "scal" and c["tree"] == "flat" and c["threads"] > 32:
                assert p is None           # one halving tree over > 32 work-items: no template
                seen_rejected += 1
                continue
            assert p is not None, d.expr
            for k in ("tile", "vw", "threads", "staged"):
                assert p[k] == c[k], (k, d.choice, p)
            if op != "scal":
                assert p["strided"] == c["strided"] and p["tree"] == c["tree"]
    assert seen_rejected > 0


def test_fig8_rules_open_every_reduction_derivation():
    d = D.derive_reduction("asum", 2048, 4, 256, True, "two", False)
    names = [s for s, _ in d.steps]
    assert names[:3] == ["r3d_partial", "r3c_split_map", "r3f_fuse_maps"]
    assert "r4e_vectorize_map" in names and "r4c_reorder" in names and "r3a_iterate" in names
    assert D.parameters(d.expr) == dict(kind="reduce", tile=2048, vw=4, threads=256,
                                        strided=True, tree="two", staged=False)


def test_library_variants_reached_and_not():
    from paper_1502_02389_gb300 import build, lift
    build.build()
    r = D.report("asum")
    assert "asum_t4096_v4_ldg_p1" in r["library_reached"]
    assert "asum_w32_t256_v8_ldg_p1" in r["library_reached"]
    assert "asum_t4096_v4_tma4_p1" in r["library_reached"]        # toLocal staging (4d)
    assert all("_c" in n for n in r["library_not_derivable"])   # only cluster stages
    assert len(D.derivable_variants("scal")) == lift.lift_variant_count(lift.OP_SCAL)
    # gemv: every variant -- a warp per row, direct (persistent or one CTA
    # per row group) or staged through shared memory (bulk or tensor
    # copies), and the rows split over CTAs
    assert D.derivable_variants("gemv") == list(range(lift.lift_variant_count(lift.OP_GEMV)))
    derived = [n for n in r["library_reached"] if n.startswith("asum_d")]
    assert len(derived) == sum(ln.startswith("LIFT_DERIVED(0,") for ln in D.emit_lines())


def test_emitted_list_is_current():
    path = os.path.join(os.path.dirname(D.__file__), "csrc", "derived_variants.inc")
    lines = [ln.strip() for ln in open(path) if ln.startswith("LIFT_DERIVED")]
    assert lines == D.emit_lines()
