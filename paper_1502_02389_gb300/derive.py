"""Rule-driven enumeration of kernel variants (arXiv 1502.02389, Sec. 6 and
Sec. 7 "Towards Automatic Derivation").

The rewrite rules of Fig. 3 (algorithmic) and Fig. 4 (OpenCL lowering) span a
space of implementations of each program of Fig. 5.  ``derive(op)`` walks
that space the way Fig. 8 derives asum: it starts from the op's high-level
expression and applies one rule at a time to a window of the current
expression, taking at every choice point each value of a small parameter
set (split sizes, work-group sizes, vector widths, the lowering of each
reorder, the shape of the in-work-group reduction tree, staging of the input
through local memory).  Each complete derivation ends in a low-level
expression; ``parameters`` reads the kernel-template parameters off that
expression, or returns None for a form that no template implements, and
``derivable_variants`` lists the library variants some derivation reaches.
The autotuner can restrict its sweep to those (``tune.py --derived``).

Besides the rules as the paper prints them, a few steps combine rules (each
names the rules it combines); ``pad`` states the reading that a reduce over
an array padded with the neutral element has the same value (used where a
tree's width is not a power of two).

The module builds expressions only; it evaluates nothing and shares no code
with any reference implementation.
"""
from __future__ import annotations

import argparse
import itertools
from dataclasses import dataclass, field
from typing import Any, Dict, Iterator, List, Optional, Sequence, Tuple

# ---------------------------------------------------------------------------
# expressions (Table 1 and Table 2 patterns, user functions)
# ---------------------------------------------------------------------------


@dataclass(frozen=True)
class Fn:
    """User function: add, abs, mult, square, id, mult_by(a), fold(f, g)
    (lambda acc, x: f(acc, g(x))), vect(n, f)."""
    name: str
    args: Tuple[Any, ...] = ()

    def __repr__(self) -> str:
        if self.name == "fold":
            return f"fold({self.args[0]!r}, {self.args[1]!r})"
        if self.name == "vect":
            return f"vectorize-{self.args[0]}({self.args[1]!r})"
        if self.name == "mult_by":
            return f"mult({self.args[0]})"
        return self.name


ADD, ABS, MULT, SQUARE, ID, SQRT = (Fn("add"), Fn("abs"), Fn("mult"), Fn("square"), Fn("id"),
                                    Fn("sqrt"))


@dataclass(frozen=True)
class Map:
    kind: str            # map | map-workgroup | map-local | map-seq | map-global
    f: Any

    def __repr__(self) -> str:
        return f"{self.kind}({self.f!r})"


@dataclass(frozen=True)
class Reduce:
    kind: str            # reduce | reduce-seq
    f: Fn
    z: Any = 0

    def __repr__(self) -> str:
        return f"{self.kind}({self.f!r}, {self.z})"


@dataclass(frozen=True)
class Split:
    n: int

    def __repr__(self) -> str:
        return f"split-{self.n}"


@dataclass(frozen=True)
class Join:
    def __repr__(self) -> str:
        return "join"


@dataclass(frozen=True)
class Reorder:
    def __repr__(self) -> str:
        return "reorder"


@dataclass(frozen=True)
class ReorderStride:
    """reorder-stride with stride s, or (s = 0) with s = len / n."""
    s: int = 0
    n: int = 0

    def __repr__(self) -> str:
        return f"reorder-stride-{self.s}" if self.s else f"reorder-stride(n={self.n})"


@dataclass(frozen=True)
class AsVector:
    n: int

    def __repr__(self) -> str:
        return f"asVector-{self.n}"


@dataclass(frozen=True)
class AsScalar:
    def __repr__(self) -> str:
        return "asScalar"


@dataclass(frozen=True)
class Iterate:
    k: int
    f: Any

    def __repr__(self) -> str:
        return f"iterate-{self.k}({self.f!r})"


@dataclass(frozen=True)
class ToLocal:
    f: Any

    def __repr__(self) -> str:
        return f"toLocal({self.f!r})"


@dataclass(frozen=True)
class Pad:
    """Pad the outer dimension to n with the reduction's neutral element."""
    n: int

    def __repr__(self) -> str:
        return f"pad-{self.n}"


@dataclass(frozen=True)
class ZipWith:
    """zip of each element (a row) with a captured vector: the dot(x) that
    gemv maps over the rows of A (Fig. 5)."""
    name: str

    def __repr__(self) -> str:
        return f"zip({self.name})"


@dataclass(frozen=True)
class C:
    """Composition fs[0] . fs[1] . ... (the last is applied first)."""
    fs: Tuple[Any, ...]

    def __repr__(self) -> str:
        return " o ".join(repr(f) for f in self.fs)


def comp(*fs) -> Any:
    flat: List[Any] = []
    for f in fs:
        flat.extend(f.fs if isinstance(f, C) else [f])
    return flat[0] if len(flat) == 1 else C(tuple(flat))


def parts(e) -> Tuple[Any, ...]:
    return e.fs if isinstance(e, C) else (e,)


# ---------------------------------------------------------------------------
# rules: each rewrites a window of consecutive functions of a composition
# ---------------------------------------------------------------------------
class NotApplicable(Exception):
    pass


def r3c_split_join(w, n):
    """Fig. 3c: map(f) -> join . map(map(f)) . split^n."""
    (m,) = w
    if not (isinstance(m, Map) and m.kind == "map"):
        raise NotApplicable
    return [Join(), Map("map", Map("map", m.f)), Split(n)]


def r3d_partial(w, n):
    """Fig. 3d: reduce(f) -> reduce(f) . part-red(f), part-red(f) ->
    join . map(part-red(f)) . split^n, part-red(f) -> reduce(f)."""
    (r,) = w
    if not (isinstance(r, Reduce) and r.kind == "reduce"):
        raise NotApplicable
    return [r, Join(), Map("map", r), Split(n)]


def r3d_partial_vectors(w, n):
    """Fig. 3d on a reduce of a vector stream seen as scalars: reduce(f) .
    asScalar -> reduce(f) . join . map(reduce(f) . asScalar) . split^n."""
    r, a = w
    if not (isinstance(r, Reduce) and r.kind == "reduce" and isinstance(a, AsScalar)):
        raise NotApplicable
    return [r, Join(), Map("map", comp(r, AsScalar())), Split(n)]


def r3b_reorder(w):
    """Fig. 3b: a reduce of a commutative f ignores the order of its input:
    reduce(f) -> reduce(f) . reorder (on a vector stream: after asScalar)."""
    if len(w) == 1 and isinstance(w[0], Reduce) and w[0].kind == "reduce":
        return [w[0], Reorder()]
    if len(w) == 2 and isinstance(w[0], Reduce) and isinstance(w[1], AsScalar):
        return [w[0], w[1], Reorder()]
    raise NotApplicable


def r3b_reorder_map(w):
    """Fig. 3b: reorder . map(f) -> map(f) . reorder."""
    o, m = w
    if not (isinstance(o, Reorder) and isinstance(m, Map)):
        raise NotApplicable
    return [m, o]


def r3c_split_map(w):
    """Fig. 3c on a mapped input: split^n . map(f) -> map(map(f)) . split^n."""
    s, m = w
    if not (isinstance(s, Split) and isinstance(m, Map) and m.kind == "map"):
        raise NotApplicable
    return [Map("map", m), s]


def r3f_fuse_maps(w):
    """Fig. 3f: map(f) . map(g) -> map(f . g)."""
    a, b = w
    if not (isinstance(a, Map) and isinstance(b, Map) and a.kind == b.kind == "map"):
        raise NotApplicable
    return [Map("map", comp(a.f, b.f))]


def r3f_fold(w):
    """Fig. 3f: reduce-seq(f, z) . map(g) -> reduce-seq(lambda acc, x. f(acc, g(x)), z)."""
    r, m = w
    if not (isinstance(r, Reduce) and r.kind == "reduce-seq" and isinstance(m, Map)
            and isinstance(m.f, Fn)):
        raise NotApplicable
    return [Reduce("reduce-seq", Fn("fold", (r.f, m.f)), r.z)]


def r3a_iterate(w, k):
    """Fig. 3a with 3d and 3b: a reduce over 2^k values halves its input k
    times, each level join . map(reduce(f)) . split^2 . reorder."""
    (r,) = w
    if not (isinstance(r, Reduce) and r.kind == "reduce"):
        raise NotApplicable
    return [Iterate(k, comp(Join(), Map("map", r), Split(2), Reorder()))]


def r_pad(w, n):
    """reduce(f, z) -> reduce(f, z) . pad-n (z neutral for f)."""
    (r,) = w
    if not isinstance(r, Reduce):
        raise NotApplicable
    return [r, Pad(n)]


def r4e_vectorize_map(w, n):
    """Fig. 4e: map(f) -> asScalar . map(vectorize-n(f)) . asVector-n."""
    (m,) = w
    if not (isinstance(m, Map) and isinstance(m.f, Fn)):
        raise NotApplicable
    return [AsScalar(), Map(m.kind, Fn("vect", (n, m.f))), AsVector(n)]


def r4e_lane_fold(w):
    """Fig. 4e with 3f and 4b on a per-thread reduce of vectors:
    reduce(+, 0) . asScalar . map(vectorize-n(g)) -> reduce-seq(+, 0) .
    asScalar . reduce-seq(vectorize-n(fold(+, g)), 0): every lane folds its
    elements, then the lanes are added (associativity and commutativity)."""
    r, a, m = w
    if not (isinstance(r, Reduce) and r.f == ADD and isinstance(a, AsScalar) and isinstance(m, Map)
            and isinstance(m.f, Fn) and m.f.name == "vect"):
        raise NotApplicable
    n, g = m.f.args
    return [Reduce("reduce-seq", ADD, r.z), AsScalar(),
            Reduce("reduce-seq", Fn("vect", (n, Fn("fold", (ADD, g)))), r.z)]


def r4a_map(w, kind):
    """Fig. 4a: map(f) -> map-workgroup | map-local | map-seq (f)."""
    (m,) = w
    if not (isinstance(m, Map) and m.kind == "map"):
        raise NotApplicable
    return [Map(kind, m.f)]


def r4b_reduce(w):
    """Fig. 4b: reduce(f, z) -> reduce-seq(f, z)."""
    (r,) = w
    if not (isinstance(r, Reduce) and r.kind == "reduce"):
        raise NotApplicable
    return [Reduce("reduce-seq", r.f, r.z)]


def r4c_reorder(w, s, n=0):
    """Fig. 4c: reorder -> id | reorder-stride (s = 0 and n = 0: id)."""
    (o,) = w
    if not isinstance(o, Reorder):
        raise NotApplicable
    return [] if (s == 0 and n == 0) else [ReorderStride(s, n)]


def r4d_to_local(w):
    """Fig. 4d: the input of a work-group copied to local memory first:
    f -> f . toLocal(map-local(id))."""
    (f,) = w
    return [f, ToLocal(Map("map-local", ID))]


# ---------------------------------------------------------------------------
# applying a rule at a place of the expression
# ---------------------------------------------------------------------------
def _body(e):
    if isinstance(e, (Map, Iterate, ToLocal)):
        return e.f
    raise NotApplicable


def _with_body(e, body):
    if isinstance(e, Map):
        return Map(e.kind, body)
    if isinstance(e, Iterate):
        return Iterate(e.k, body)
    if isinstance(e, ToLocal):
        return ToLocal(body)
    raise NotApplicable


def rewrite(e, where: Sequence[Tuple[int, ...]], start: int, length: int, rule, *args):
    """Apply ``rule`` to the window fs[start:start+length] of the
    composition reached by descending through ``where``: each step (i,)
    takes element i of a composition and enters the body of that map,
    iterate or toLocal."""
    if where:
        (i,) = where[0]
        fs = list(parts(e))
        fs[i] = _with_body(fs[i], rewrite(_body(fs[i]), where[1:], start, length, rule, *args))
        return comp(*fs)
    fs = list(parts(e))
    if start < 0 or start + length > len(fs):
        raise NotApplicable
    new = rule(tuple(fs[start:start + length]), *args)
    return comp(*(fs[:start] + list(new) + fs[start + length:]))


@dataclass
class Derivation:
    op: str
    expr: Any
    steps: List[Tuple[str, Any]] = field(default_factory=list)
    choice: Dict[str, Any] = field(default_factory=dict)

    def apply(self, where, start, length, rule, *args) -> "Derivation":
        self.expr = rewrite(self.expr, where, start, length, rule, *args)
        self.steps.append((rule.__name__, args))
        return self


# ---------------------------------------------------------------------------
# the programs (Fig. 5) and the derivation strategies
# ---------------------------------------------------------------------------
REDUCTIONS = {"asum": ABS, "dot": MULT, "nrm2": SQUARE, "sum": ID}
MAPS = {"scal": Fn("mult_by", ("a",)), "axpy": Fn("axpy", ("a",))}

TILES = (256, 512, 1024, 2048, 4096, 8192)
WG_SIZES = (32, 64, 128, 256, 512, 1024)
WIDTHS = (1, 2, 4, 8)


GEMV_ROWS = (1, 2, 4, 8, 16, 32)     # rows per work-group (a warp each)
GEMV_N = 512                          # the row length the gemv derivations are written for


def program(op: str):
    """High-level expression of an op (Fig. 5); dot and axpy take the
    zipped pair of their inputs; gemv's z = join . map(scal(a) . dot(x))
    over the rows of A."""
    if op in REDUCTIONS:
        return comp(Reduce("reduce", ADD, 0), Map("map", REDUCTIONS[op]))
    if op in MAPS:
        return Map("map", MAPS[op])
    if op == "gemv":
        row = comp(Map("map", Fn("mult_by", ("a",))), Reduce("reduce", ADD, 0), Map("map", MULT),
                   ZipWith("x"))
        return comp(Join(), Map("map", row))
    raise KeyError(op)


def _log2(x: int) -> int:
    k = x.bit_length() - 1
    return k if (1 << k) == x else -1


def derive_reduction(op: str, tile: int, vw: int, threads: int, strided: bool, tree: str,
                     staged: bool) -> Derivation:
    """One derivation of a reduction (asum, dot, nrm2, sum): tile elements
    per work-group, vw-wide vectors, threads work-items each folding
    J = tile / (vw threads) vectors (taken strided or as a contiguous run),
    the work-group tree ("warp": one halving tree over 32 work-items; "two":
    halving trees over each 32 work-items, then over their results padded to
    32; "flat": one halving tree over all work-items), input staged through
    local memory or not."""
    J = tile // (vw * threads)
    if J < 1 or J * vw * threads != tile:
        raise NotApplicable
    d = Derivation(op, program(op), choice=dict(tile=tile, vw=vw, threads=threads,
                                                strided=strided, tree=tree, staged=staged))
    # reduce . map(g)  ->  reduce . join . map(reduce . map(g)) . split^tile
    d.apply((), 0, 1, r3d_partial, tile)            # R . join . map(R) . split . map(g)
    d.apply((), 3, 2, r3c_split_map)                # R . join . map(R) . map(map(g)) . split
    d.apply((), 2, 2, r3f_fuse_maps)                # R . join . map(R . map(g)) . split
    W = ((2,),)                                     # inside the work-group's map
    _lower_workgroup(d, W, vw, J, threads, strided, tree)
    if staged:
        n = len(parts(_at(d.expr, W)))
        d.apply(W, n - 1, 1, r4d_to_local)
    d.apply((), 2, 1, r4a_map, "map-workgroup")
    d.apply((), 0, 1, r4b_reduce)                   # the outer reduce over the work-groups
    if op == "nrm2":
        d.expr = comp(Map("map-seq", SQRT), d.expr)
        d.steps.append(("sqrt of the sum (program)", ()))
    return d


def _at(e, where):
    """The composition reached by descending through ``where`` (as in
    ``rewrite``)."""
    for (i,) in where:
        e = _body(parts(e)[i])
    return e


def _lower_workgroup(d: Derivation, W, vw: int, J: int, threads: int, strided: bool, tree: str):
    """The work-group body at W, reduce . map(g) over its tile, lowered: the
    tile vectorised (vw > 1), reordered and split among `threads`
    work-items that fold J elements (vectors) each with g fused in, then the
    work-group tree over their results."""
    if vw > 1:
        d.apply(W, 1, 1, r4e_vectorize_map, vw)     # R . asScalar . map(vect g) . asVector
        d.apply(W, 0, 2, r3b_reorder)               # R . asScalar . reorder . ...
        d.apply(W, 0, 2, r3d_partial_vectors, J)    # R . join . map(R . asScalar) . split^J . reorder . map(vg) . asVector
        d.apply(W, 4, 2, r3b_reorder_map)           # ... split^J . map(vg) . reorder . asVector
        d.apply(W, 3, 2, r3c_split_map)             # ... map(map(vg)) . split^J . reorder . asVector
        d.apply(W, 2, 2, r3f_fuse_maps)             # R . join . map(R . asScalar . map(vg)) . split^J . reorder . asVector
        d.apply(W + ((2,),), 0, 3, r4e_lane_fold)   # thread: reduce-seq(+) . asScalar . reduce-seq(vect(fold))
    else:
        d.apply(W, 0, 1, r3b_reorder)               # R . reorder . map(g)
        d.apply(W, 0, 1, r3d_partial, J)            # R . join . map(R) . split^J . reorder . map(g)
        d.apply(W, 4, 2, r3b_reorder_map)           # ... split^J . map(g) . reorder
        d.apply(W, 3, 2, r3c_split_map)             # ... map(map(g)) . split^J . reorder
        d.apply(W, 2, 2, r3f_fuse_maps)             # R . join . map(R . map(g)) . split^J . reorder
        d.apply(W + ((2,),), 0, 1, r4b_reduce)      # thread: reduce-seq(+) . map(g)
        d.apply(W + ((2,),), 0, 2, r3f_fold)        # thread: reduce-seq(fold(+, g))
    # the thread order: reorder -> reorder-stride^threads (strided) | id (contiguous runs)
    body = parts(_at(d.expr, W))
    ro = [i for i, f in enumerate(body) if isinstance(f, Reorder)][0]
    d.apply(W, ro, 1, r4c_reorder, threads if strided else 0)
    d.apply(W, 2, 1, r4a_map, "map-local")          # threads
    # the work-group tree over the threads' results (element 0 of the body)
    k = _log2(threads)
    if k < 0:
        raise NotApplicable
    if tree == "flat" or threads == 32:
        if tree == "two":
            raise NotApplicable
        d.apply(W, 0, 1, r3a_iterate, k)
        _lower_tree(d, W + ((0,),))
    elif tree == "two":
        d.apply(W, 0, 1, r3d_partial, 32)           # R . join . map(R) . split^32 over the threads
        d.apply(W + ((2,),), 0, 1, r3a_iterate, 5)  # each 32: a halving tree
        _lower_tree(d, W + ((2,), (0,)))
        # the map over the 32-groups stays a map: the OpenCL patterns have no
        # level between work-group and work-item (on the GPU it is the warp)
        d.apply(W, 0, 1, r_pad, 32)                 # the W results padded to 32
        d.apply(W, 0, 1, r3a_iterate, 5)
        _lower_tree(d, W + ((0,),))
    else:
        raise NotApplicable


def _lower_tree(d: Derivation, it_where):
    """Inside iterate(join . map(reduce) . split-2 . reorder): map ->
    map-local, reduce -> reduce-seq, reorder -> reorder-stride(n = 2)
    (pairs j and j + len/2: a halving tree)."""
    d.apply(it_where, 1, 1, r4a_map, "map-local")
    d.apply(it_where + ((1,),), 0, 1, r4b_reduce)
    d.apply(it_where, 3, 1, r4c_reorder, 0, 2)


def derive_map(op: str, tile: int, vw: int, threads: int, staged: bool) -> Derivation:
    """One derivation of a map (scal, axpy): the Fig. 2b form
    join . map-workgroup(asScalar . join . map-local(map-seq(vectorize(f)))
    . split^J . asVector) . split^tile."""
    J = tile // (vw * threads)
    if J < 1 or J * vw * threads != tile:
        raise NotApplicable
    d = Derivation(op, program(op), choice=dict(tile=tile, vw=vw, threads=threads, staged=staged))
    d.apply((), 0, 1, r3c_split_join, tile)         # join . map(map(f)) . split^tile
    W = ((1,),)
    if vw > 1:
        d.apply(W, 0, 1, r4e_vectorize_map, vw)     # asScalar . map(vect f) . asVector
        d.apply(W, 1, 1, r3c_split_join, J)         # asScalar . join . map(map(vf)) . split^J . asVector
        d.apply(W + ((2,),), 0, 1, r4a_map, "map-seq")
        d.apply(W, 2, 1, r4a_map, "map-local")
    else:
        d.apply(W, 0, 1, r3c_split_join, J)         # join . map(map(f)) . split^J
        d.apply(W + ((1,),), 0, 1, r4a_map, "map-seq")
        d.apply(W, 1, 1, r4a_map, "map-local")
    if staged:
        n = len(parts(_body(parts(d.expr)[1])))
        d.apply(W, n - 1, 1, r4d_to_local)
    d.apply((), 1, 1, r4a_map, "map-workgroup")
    return d


def derive_gemv(rows: int, vw: int, strided: bool, staged: bool = False,
                n: int = GEMV_N) -> Derivation:
    """One derivation of gemv's z (Fig. 5) for rows of n elements, the form of
    the warp-per-row kernels: the rows split into work-groups of `rows`,
    each row's dot done by 32 work-items (a warp; like the 32-groups of a
    two-level reduction tree, the map over a work-group's rows stays a
    plain map) that each fold J = n / (32 vw) vectors of the row zipped with
    x (taken strided or as a contiguous run), then a halving tree over the
    32 partial sums, then the scaling by a.  Staged: the zipped row (A's row
    and x) is copied to local memory first (Fig. 4d), the form of the
    bulk-copy and tensor-copy kernels, which stream it through a ring of
    shared-memory stages."""
    J = n // (32 * vw)
    if J < 1 or J * 32 * vw != n:
        raise NotApplicable
    d = Derivation("gemv", program("gemv"),
                   choice=dict(rows=rows, vw=vw, strided=strided, staged=staged, n=n))
    d.apply((), 1, 1, r3c_split_join, rows)         # join . join . map(map(row)) . split^rows
    d.apply((), 2, 1, r4a_map, "map-workgroup")
    R = ((2,), (0,))                                # the row: map(a) . reduce . map(mult) . zip(x)
    if vw > 1:
        d.apply(R, 2, 1, r4e_vectorize_map, vw)     # map(a) . R . asScalar . map(vect mult) . asVector . zip
        d.apply(R, 1, 2, r3b_reorder)               # ... R . asScalar . reorder . map(vect) ...
        d.apply(R, 1, 2, r3d_partial_vectors, J)    # map(a) . R . join . map(R . asScalar) . split^J . reorder . map(vect) . asVector . zip
        d.apply(R, 5, 2, r3b_reorder_map)           # ... split^J . map(vect) . reorder . asVector . zip
        d.apply(R, 4, 2, r3c_split_map)             # ... map(map(vect)) . split^J . reorder ...
        d.apply(R, 3, 2, r3f_fuse_maps)             # map(a) . R . join . map(R . asScalar . map(vect)) . split^J ...
        d.apply(R + ((3,),), 0, 3, r4e_lane_fold)   # work-item: reduce-seq(+) . asScalar . reduce-seq(vect(fold))
    else:
        d.apply(R, 1, 1, r3b_reorder)               # map(a) . R . reorder . map(mult) . zip
        d.apply(R, 1, 1, r3d_partial, J)            # map(a) . R . join . map(R) . split^J . reorder . map(mult) . zip
        d.apply(R, 5, 2, r3b_reorder_map)           # ... split^J . map(mult) . reorder . zip
        d.apply(R, 4, 2, r3c_split_map)             # ... map(map(mult)) . split^J . reorder . zip
        d.apply(R, 3, 2, r3f_fuse_maps)             # map(a) . R . join . map(R . map(mult)) . split^J . reorder . zip
        d.apply(R + ((3,),), 0, 1, r4b_reduce)      # work-item: reduce-seq(+) . map(mult)
        d.apply(R + ((3,),), 0, 2, r3f_fold)        # work-item: reduce-seq(fold(+, mult))
    d.apply(R, 5, 1, r4c_reorder, 32 if strided else 0)
    d.apply(R, 3, 1, r4a_map, "map-local")          # the 32 work-items of the row
    d.apply(R, 1, 1, r3a_iterate, 5)                # the halving tree over their 32 sums
    _lower_tree(d, R + ((1,),))
    d.apply(R, 0, 1, r4a_map, "map-seq")            # a * (the row's dot)
    if staged:                                      # ... . toLocal(map-local(id)) . zip(x)
        n_row = len(parts(_body(parts(_body(parts(d.expr)[2]))[0])))
        d.apply(R, n_row - 2, 1, r4d_to_local)
    return d


GEMV_SPLIT_N = 8192          # the row length the split-row derivations are written for
GEMV_SEGMENTS = (1024, 2048, 4096)


def derive_gemv_split(threads: int, vw: int, strided: bool, seg: int,
                      n: int = GEMV_SPLIT_N) -> Derivation:
    """One derivation of gemv's z with each row's reduce split by Fig. 3d into
    S = n / seg segments of seg elements, one work-group per segment lowered
    like a reduction's work-group (threads work-items folding strided or
    contiguous vectors, the two-level tree), then the combine of the S
    partials, padded to 32, by a halving tree (the warp of the second
    launch: its own work-group, so the map of that tree stays a plain map),
    then the scaling by a.  The rows stay a plain map (the grid's second
    dimension)."""
    J = seg // (vw * threads)
    S = n // seg
    if J < 1 or J * vw * threads != seg or S * seg != n or S > 32 or threads <= 32:
        raise NotApplicable
    d = Derivation("gemv", program("gemv"),
                   choice=dict(split=True, threads=threads, vw=vw, strided=strided, seg=seg, n=n))
    R = ((1,),)                                     # the row: map(a) . reduce . map(mult) . zip(x)
    d.apply(R, 1, 1, r3d_partial, seg)              # map(a) . R . join . map(R) . split^seg . map(mult) . zip
    d.apply(R, 4, 2, r3c_split_map)                 # ... map(R) . map(map(mult)) . split^seg . zip
    d.apply(R, 3, 2, r3f_fuse_maps)                 # map(a) . R . join . map(R . map(mult)) . split^seg . zip
    _lower_workgroup(d, R + ((3,),), vw, J, threads, strided, "two")
    d.apply(R, 3, 1, r4a_map, "map-workgroup")      # a work-group per segment
    d.apply(R, 1, 1, r_pad, 32)                     # the S partials padded to 32
    d.apply(R, 1, 1, r3a_iterate, 5)                # the combine's halving tree
    d.apply(R + ((1,), (1,)), 0, 1, r4b_reduce)
    d.apply(R + ((1,),), 3, 1, r4c_reorder, 0, 2)
    d.apply(R, 0, 1, r4a_map, "map-seq")            # a * (the row's dot)
    return d


def derive(op: str) -> Iterator[Derivation]:
    """Every derivation of an op over the parameter sets."""
    if op in REDUCTIONS:
        for tile, vw, t, strided, tree, staged in itertools.product(
                TILES, WIDTHS, WG_SIZES, (True, False), ("warp", "two", "flat"), (False, True)):
            if (tree == "warp") != (t == 32):      # over 32 work-items "flat" is "warp"
                continue
            try:
                yield derive_reduction(op, tile, vw, t, strided, tree, staged)
            except NotApplicable:
                continue
    elif op in MAPS:
        for tile, vw, t, staged in itertools.product(TILES, WIDTHS, WG_SIZES, (False, True)):
            try:
                yield derive_map(op, tile, vw, t, staged)
            except NotApplicable:
                continue
    elif op == "gemv":
        for rows, vw, strided, staged in itertools.product(GEMV_ROWS, WIDTHS, (True, False),
                                                            (False, True)):
            try:
                yield derive_gemv(rows, vw, strided, staged)
            except NotApplicable:
                continue
        for threads, vw, strided, seg in itertools.product(WG_SIZES, WIDTHS, (True, False),
                                                            GEMV_SEGMENTS):
            try:
                yield derive_gemv_split(threads, vw, strided, seg)
            except NotApplicable:
                continue
    else:
        raise KeyError(op)


# ---------------------------------------------------------------------------
# reading kernel parameters off a low-level expression
# ---------------------------------------------------------------------------
def _is_halving(e, levels: int, kind: str = "map-local") -> bool:
    if not (isinstance(e, Iterate) and e.k == levels):
        return False
    b = parts(e.f)
    return (len(b) == 4 and isinstance(b[0], Join) and isinstance(b[1], Map)
            and b[1].kind == kind and isinstance(b[1].f, Reduce)
            and b[1].f.kind == "reduce-seq" and b[1].f.f == ADD and isinstance(b[2], Split)
            and b[2].n == 2 and b[3] == ReorderStride(0, 2))


def parameters(e) -> Optional[Dict[str, Any]]:
    """Kernel-template parameters of a low-level expression, or None when
    no template implements it.  Reductions: reduce-seq . join .
    map-workgroup(TREE . join . map-local(THREAD) . split^J . [reorder-stride^T]
    . [asVector^vw] . [toLocal(map-local(id))]) . split^tile, TREE a halving
    tree over 32 work-items or halving trees over 32s then over their padded
    results.  Maps: join . map-workgroup([asScalar .] join .
    map-local(map-seq(f)) . split^J [. asVector^vw] [. toLocal(...)]) . split^tile."""
    fs = list(parts(e))
    if fs and isinstance(fs[0], Map) and fs[0].kind == "map-seq":      # nrm2's sqrt
        fs = fs[1:]
    # --- maps
    if len(fs) == 3 and isinstance(fs[0], Join) and isinstance(fs[1], Map) \
            and fs[1].kind == "map-workgroup" and isinstance(fs[2], Split):
        b = list(parts(fs[1].f))
        staged = bool(b) and isinstance(b[-1], ToLocal)
        if staged:
            b = b[:-1]
        vw = 1
        if b and isinstance(b[0], AsScalar):
            if not (isinstance(b[-1], AsVector)):
                return None
            vw = b[-1].n
            b = b[1:-1]
        if not (len(b) == 3 and isinstance(b[0], Join) and isinstance(b[1], Map)
                and b[1].kind == "map-local" and isinstance(b[1].f, Map)
                and b[1].f.kind == "map-seq" and isinstance(b[2], Split)):
            return None
        J = b[2].n
        return dict(kind="map", tile=fs[2].n, vw=vw, threads=fs[2].n // (vw * J), staged=staged)
    # --- gemv: join . join . map-workgroup(map(ROW)) . split^rows, ROW =
    # map-seq(a) . TREE32 . join . map-local(THREAD) . split^J
    #   [. reorder-stride^32] [. asVector^vw] . zip(x)
    if (len(fs) == 4 and isinstance(fs[0], Join) and isinstance(fs[1], Join)
            and isinstance(fs[2], Map) and fs[2].kind == "map-workgroup"
            and isinstance(fs[2].f, Map) and fs[2].f.kind == "map" and isinstance(fs[3], Split)):
        r = list(parts(fs[2].f.f))
        if not (r and isinstance(r[-1], ZipWith)):
            return None
        r = r[:-1]
        staged = isinstance(r[-1], ToLocal)
        if staged:
            r = r[:-1]
        vw = r.pop().n if isinstance(r[-1], AsVector) else 1
        strided = isinstance(r[-1], ReorderStride)
        if strided and r.pop().s != 32:
            return None
        if not (len(r) == 5 and isinstance(r[0], Map) and r[0].kind == "map-seq"
                and _is_halving(r[1], 5) and isinstance(r[2], Join) and isinstance(r[3], Map)
                and r[3].kind == "map-local" and isinstance(r[4], Split)):
            return None
        return dict(kind="gemv", rows=fs[3].n, vw=vw, lanes=32, strided=strided, staged=staged)
    # --- gemv with split rows: join . map(ROW), ROW = map-seq(a) . COMBINE
    # . pad-32 . join . map-workgroup(SEGMENT) . split^L . zip(x), COMBINE a
    # halving tree over 32 (the second launch's warp), SEGMENT a reduction
    # work-group body
    if (len(fs) == 2 and isinstance(fs[0], Join) and isinstance(fs[1], Map)
            and fs[1].kind == "map"):
        r = list(parts(fs[1].f))
        if not (len(r) == 7 and isinstance(r[0], Map) and r[0].kind == "map-seq"
                and _is_halving(r[1], 5, "map") and r[2] == Pad(32) and isinstance(r[3], Join)
                and isinstance(r[4], Map) and r[4].kind == "map-workgroup"
                and isinstance(r[5], Split) and isinstance(r[6], ZipWith)):
            return None
        w = _workgroup_params(list(parts(r[4].f)), r[5].n)
        if w is None or w["tree"] != "two" or w["staged"]:
            return None
        return dict(kind="gemv_split", threads=w["threads"], vw=w["vw"], strided=w["strided"])
    # --- reductions
    if not (len(fs) == 4 and isinstance(fs[0], Reduce) and fs[0].kind == "reduce-seq"
            and isinstance(fs[1], Join) and isinstance(fs[2], Map)
            and fs[2].kind == "map-workgroup" and isinstance(fs[3], Split)):
        return None
    w = _workgroup_params(list(parts(fs[2].f)), fs[3].n)
    return None if w is None else dict(kind="reduce", **w)


def _workgroup_params(b, tile: int) -> Optional[Dict[str, Any]]:
    """(tile, vw, threads, strided, tree, staged) of a reduction's work-group
    body TREE . join . map-local(THREAD) . split^J [. reorder-stride^T]
    [. asVector^vw] [. toLocal(map-local(id))] over `tile` elements."""
    staged = isinstance(b[-1], ToLocal)
    if staged:
        b = b[:-1]
    vw = 1
    if isinstance(b[-1], AsVector):
        vw = b.pop().n
    strided = isinstance(b[-1], ReorderStride)
    stride = b.pop() if strided else None
    # tree . join . map-local(thread) . split^J
    if len(b) < 4 or not isinstance(b[-1], Split) or not isinstance(b[-3], Join):
        return None
    J = b[-1].n
    thread = b[-2]
    if not (isinstance(thread, Map) and thread.kind == "map-local"):
        return None
    threads = tile // (vw * J)
    if strided and stride.s != threads:
        return None
    tree = b[:-3]
    if len(tree) == 1 and _is_halving(tree[0], 5) and threads == 32:
        form = "warp"
    elif (len(tree) == 5 and _is_halving(tree[0], 5) and isinstance(tree[1], Pad)
          and tree[1].n == 32 and isinstance(tree[2], Join) and isinstance(tree[3], Map)
          and tree[3].kind == "map" and _is_halving(tree[3].f, 5)
          and isinstance(tree[4], Split) and tree[4].n == 32 and 32 < threads <= 1024):
        form = "two"
    else:
        return None        # e.g. one halving tree over more than 32 work-items
    return dict(tile=tile, vw=vw, threads=threads, strided=strided, tree=form, staged=staged)


# ---------------------------------------------------------------------------
# the library's variants reached by derivations
# ---------------------------------------------------------------------------
OP_IDS = {"asum": 0, "dot": 1, "scal": 2, "gemv": 3, "nrm2": 8, "sum": 9, "axpy": 10}


def variant_key(info: Dict[str, Any]) -> Optional[Tuple]:
    """The derivation-visible parameters of a library variant (None for a
    variant no pattern expresses, e.g. a thread-block-cluster stage)."""
    if info["cluster"] > 1:
        return None
    if info["op"] in (OP_IDS["scal"], OP_IDS["axpy"]):
        return ("map", info["tile"], info["vw"], info["threads"], info["stages"] > 0)
    if info["op"] == OP_IDS["gemv"]:
        # a warp per row, direct or staged through shared memory (bulk or
        # tensor copies: info tree 3); the split-row form, which spreads a
        # row over several CTAs, is not among the enumerated derivations
        if info["lanes"] == 32 and info["tree"] in (0, 3):
            return ("gemv", info["rows"], info["vw"], bool(info["stride"]), info["stages"] > 0)
        if info["lanes"] == info["threads"] > 32 and info["rows"] == 1:     # rows split over CTAs
            return ("gemv_split", info["threads"], info["vw"], bool(info["stride"]))
        return None
    tree = {0: "warp", 1: "two"}.get(info["tree"])
    return ("reduce", info["tile"], info["vw"], info["threads"], bool(info["stride"]), tree,
            info["stages"] > 0)


def param_key(p: Dict[str, Any]) -> Tuple:
    if p["kind"] == "map":
        return ("map", p["tile"], p["vw"], p["threads"], p["staged"])
    if p["kind"] == "gemv":
        return ("gemv", p["rows"], p["vw"], p["strided"], p["staged"])
    if p["kind"] == "gemv_split":
        return ("gemv_split", p["threads"], p["vw"], p["strided"])
    return ("reduce", p["tile"], p["vw"], p["threads"], p["strided"], p["tree"], p["staged"])


def enumerate_op(op: str):
    """(derivations, {key: params} of the implementable ones, rejected count)."""
    ders = list(derive(op))
    keys: Dict[Tuple, Dict[str, Any]] = {}
    rejected = 0
    for d in ders:
        p = parameters(d.expr)
        if p is None:
            rejected += 1
        else:
            keys.setdefault(param_key(p), p)
    return ders, keys, rejected


def derivable_variants(op: str) -> List[int]:
    """Ids of the library variants of ``op`` whose parameters a derivation
    reaches."""
    from . import lift
    _, keys, _ = enumerate_op(op)
    out = []
    for v in range(lift.lift_variant_count(OP_IDS[op])):
        k = variant_key(lift.lift_variant_describe(OP_IDS[op], v))
        if k is not None and k in keys:
            out.append(v)
    return out


def report(op: str) -> Dict[str, Any]:
    from . import lift
    ders, keys, rejected = enumerate_op(op)
    lib = {}
    for v in range(lift.lift_variant_count(OP_IDS[op])):
        info = lift.lift_variant_describe(OP_IDS[op], v)
        lib[v] = (info["name"], variant_key(info))
    reached = [name for name, k in lib.values() if k is not None and k in keys]
    outside = [name for name, k in lib.values() if k is None or k not in keys]
    lib_keys = {k for _, k in lib.values()}
    missing = sorted(k for k in keys if k not in lib_keys)
    return {"op": op, "derivations": len(ders), "implementable": len(keys), "rejected": rejected,
            "library_reached": reached, "library_not_derivable": outside,
            "derivable_not_instantiated": missing}


# Parameter sets instantiated from the enumeration (reduce_derived.cu): the
# implementable two-level-tree, strided, directly loaded forms with work-group
# sizes the hand-picked list (32 and 256 work-items) leaves out.
EMIT_THREADS = (128, 512)
EMIT_TILES = (1024, 2048, 4096)
EMIT_WIDTHS = (4, 8)


def emit_lines() -> List[str]:
    out = []
    for op, code in (("asum", 0), ("dot", 1)):
        _, keys, _ = enumerate_op(op)
        for k in sorted(keys):
            p = keys[k]
            if (p["tree"] == "two" and p["strided"] and not p["staged"]
                    and p["threads"] in EMIT_THREADS and p["tile"] in EMIT_TILES
                    and p["vw"] in EMIT_WIDTHS):
                name = f"d{p['threads']}_t{p['tile']}_v{p['vw']}"
                out.append(f'LIFT_DERIVED({code}, {p["threads"]}, {p["tile"]}, {p["vw"]}, true, 0, '
                           f'"{name}")')
    return out


def emit(path: str) -> int:
    lines = emit_lines()
    with open(path, "w") as f:
        f.write("// Written by `python -m paper_1502_02389_gb300.derive --emit`: parameter sets\n"
                "// (op 0 asum / 1 dot, work-items, tile, vector width, strided, stages, name)\n"
                "// reached by rule derivations of the Fig. 5 programs.\n")
        for ln in lines:
            f.write(ln + "\n")
    return len(lines)


def main():
    ap = argparse.ArgumentParser(description="enumerate rule derivations of an op")
    ap.add_argument("--op", default="asum", choices=sorted(OP_IDS))
    ap.add_argument("--show", type=int, default=1, help="print this many derivations")
    ap.add_argument("--emit", action="store_true",
                    help="write csrc/derived_variants.inc (then rebuild the library)")
    a = ap.parse_args()
    if a.emit:
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc",
                            "derived_variants.inc")
        print(f"{emit(path)} parameter sets written to {path}")
        return
    ders, keys, rejected = enumerate_op(a.op)
    for d in ders[:a.show]:
        print(d.choice)
        for name, args in d.steps:
            print("   ", name, args)
        print("  =", d.expr)
        print("  ->", parameters(d.expr))
    r = report(a.op)
    print(f"{r['derivations']} derivations, {r['implementable']} implementable parameter sets, "
          f"{r['rejected']} rejected")
    print(f"library variants reached: {len(r['library_reached'])}; not derivable: "
          f"{r['library_not_derivable']}")
    print(f"derivable, not instantiated: {len(r['derivable_not_instantiated'])}")


if __name__ == "__main__":
    main()
