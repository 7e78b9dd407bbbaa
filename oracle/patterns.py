"""Interpreter and type checker of the pattern language (arXiv 1502.02389, Sec. 3).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

An expression is a tree of frozen dataclasses.  ``Compose((f, g, h))`` is
f . g . h, so ``h`` is applied first (Sec. 2: (f . g)(x) = f(g(x))).  Every
value is an array; a primitive is an array of length 1 (Sec. 3, "all types
are arrays").  Sizes live in the type (Sec. 3.1, "Zip and Split/Join";
Sec. 7.1), so ``infer`` rejects ill-typed expressions before ``evaluate``
runs them.

Value semantics, one per pattern (Table 1 and Table 2):

* map(f), map-workgroup(f), map-local(f), map-global(f), map-seq(f):
  apply f to every element of the outermost dimension.  The four OpenCL maps
  have the value semantics of map (Table 2, "identical to map(f)"); they
  differ only in the thread-hierarchy rule that ``infer`` checks (Sec. 4.2,
  "Maps": a map-local is legal only inside a map-workgroup).
* reduce(f, z), reduce-seq(f, z): the left fold from z --
  acc = z; for each element e in order: acc = f(acc, e); result [acc]
  (Sec. 3.2, "Sequential Map and Reduce").  reduce requires f associative and
  commutative (Sec. 3.1), so any association order is a correct result; the
  interpreter evaluates the left fold.
* part-red(f, z): n elements to m with 1 <= m < n (Sec. 4.1).  Its value is
  fixed only once a derivation of Fig. 3d picks a form; the interpreter uses
  the first form, part-red -> reduce (m = 1), the same step Fig. 8 takes from
  (6) to (7).
* zip: two arrays of equal length to an array of pairs (Table 1).
* split^n: T[m] -> T[m/n][n]; a type error unless n divides m (sizes are part
  of the type; the paper never splits a non-multiple).
* join: T[m][n] -> T[m*n].
* iterate^n(f): f applied n times; f^0 = id, f^(n+1) = f^n . f (Sec. 3.1).
* reorder: "the order does not matter" (Sec. 3.1).  Any permutation is a
  valid value; the interpreter returns the input order (identity), which is
  one of the two lowerings of Fig. 4c.
* reorder-stride^s: out[i] = in[i / n + s * (i mod n)] with n * s = len
  (Sec. 3.2, "Reorder-stride").  Fig. 9 prints it without s; ``ReorderStride``
  therefore takes either s or n (the other follows from the length).
* toLocal(f), toGlobal(f): f's value, stored in another address space
  (Sec. 3.2, "Local/Global"); the type records the space.
* asVector^n: T[..][m] -> Tn[..][m/n]; asScalar: Tn[..][m] -> T[..][m*n]
  (Table 2).  A vector element is stored as a trailing lane axis.
* vect^n(f): f applied lane-wise to vectors of width n (Table 2).

Two nodes are not patterns of the paper and say so where they are used:
``ZipWith`` zips the input with a captured array (the partial application
dot(x) of Fig. 5), and ``PadTo`` appends the neutral element of a reduction
(used to state what a GPU kernel computes on a ragged tail).

Arithmetic modes.  ``mode='f64'`` evaluates every user function in IEEE
double precision (the oracle proper).  ``mode='f32'`` evaluates every user
function in IEEE single precision with round-to-nearest-even after each
operation, except ``add64`` and ``to_f64`` (FP64 combine steps); it
states, operation by operation, what an fp32 kernel built from the same
low-level expression computes.  ``mode='int'`` keeps integers (Fig. 2).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Any, Dict, Optional, Tuple, Union

import numpy as np


class PatternTypeError(TypeError):
    """The expression is ill-typed for its input (Sec. 7.1: the type system
    prevents the user from producing incorrect expressions)."""


# ============================================================================
# User functions (Sec. 3: they operate on primitives; Fig. 5 defines add,
# mult and abs)
# ============================================================================
@dataclass(frozen=True)
class UserFun:
    """A user function on primitives.  ``name`` selects its arithmetic,
    ``params`` holds partially applied arguments or sub-functions."""

    name: str
    params: Tuple[Any, ...] = ()

    def __repr__(self) -> str:  # compact, paper-like printing
        if self.name == "mult_by":
            return f"mult({self.params[0]!r})"
        if self.name == "fold":
            f, g = self.params
            return f"(lambda acc,x: {f!r}(acc, {g!r}(x)))"
        if self.name == "compose":
            return f"({self.params[0]!r} . {self.params[1]!r})"
        return self.name


ARITY = {"abs": 1, "id": 1, "mul3": 1, "mult_by": 1, "to_f32": 1, "to_f64": 1,
         "neg": 1, "add": 2, "add64": 2, "mult": 2, "fold": 2, "compose": 1,
         "square": 1, "sqrt64": 1}

abs_ = UserFun("abs")          # Fig. 5: abs(x) = if (x < 0) -x else x
id_ = UserFun("id")
add = UserFun("add")           # Fig. 5: add(x, y) = x + y
mult = UserFun("mult")         # Fig. 5: mult(x, y) = x * y
mul3 = UserFun("mul3")         # Fig. 2a: mul3(x) = x * 3
neg = UserFun("neg")
add64 = UserFun("add64")       # x + y always in FP64 (combine steps)
to_f32 = UserFun("to_f32")     # round to fp32 (the store of an fp32 result)
to_f64 = UserFun("to_f64")     # widen to fp64 (exact)
square = UserFun("square")     # x * x
sqrt64 = UserFun("sqrt64")     # correctly rounded square root, always in FP64


def mult_by(a) -> UserFun:
    """mult(a): mult with its first argument bound (Fig. 5, scal)."""
    return UserFun("mult_by", (a,))


def fold(f: UserFun, g: UserFun) -> UserFun:
    """lambda acc, x: f(acc, g(x)) -- the fused reduction function that the
    second fusion rule of Fig. 3f builds."""
    return UserFun("fold", (f, g))


def compose_fun(f: UserFun, g: UserFun) -> UserFun:
    """f . g on primitives (the first fusion rule of Fig. 3f on user functions)."""
    return UserFun("compose", (f, g))


absAndPlus = fold(add, abs_)   # Fig. 9: lambda acc, a: acc + abs(a)


def arity(f) -> int:
    if isinstance(f, Vect):
        return arity(f.f)
    return ARITY[f.name]


# ============================================================================
# Expression nodes
# ============================================================================
class Expr:
    """Base class of pattern nodes."""


@dataclass(frozen=True)
class Compose(Expr):
    fs: Tuple[Any, ...]

    def __repr__(self) -> str:
        return " o ".join(repr(f) for f in self.fs)


@dataclass(frozen=True)
class Map(Expr):
    f: Any
    kind: str = "map"   # map | map-workgroup | map-local | map-global | map-seq

    def __repr__(self) -> str:
        return f"{self.kind}({self.f!r})"


def MapWorkgroup(f):
    return Map(f, "map-workgroup")


def MapLocal(f):
    return Map(f, "map-local")


def MapGlobal(f):
    return Map(f, "map-global")


def MapSeq(f):
    return Map(f, "map-seq")


MAP_KINDS = ("map", "map-workgroup", "map-local", "map-global", "map-seq")


@dataclass(frozen=True)
class Reduce(Expr):
    f: Any
    z: Any = 0
    kind: str = "reduce"   # reduce | reduce-seq | part-red

    def __repr__(self) -> str:
        return f"{self.kind}({self.f!r}, {self.z!r})"


def ReduceSeq(f, z=0):
    return Reduce(f, z, "reduce-seq")


def PartRed(f, z=0):
    return Reduce(f, z, "part-red")


def ReduceSeqComp(f=None):
    """reduce-seq with a (sum, compensation) accumulator: Neumaier's
    compensated summation (Neumaier 1974).  For each element t in order:
    s' = s + t; c = c + ((s - s') + t if |s| >= |t| else (t - s') + s);
    s = s'; the result is s + c (s itself when s is not finite, so an Inf
    among the terms stays Inf).  In exact arithmetic this is reduce(add, 0);
    in fp32 its error is about 2u|sum| whatever the number of elements.
    ``f`` is add, or vect^n(add) to sum vectors lane by lane."""
    return Reduce(add if f is None else f, 0, "reduce-seq-comp")


@dataclass(frozen=True)
class Zip(Expr):
    """zip(a, b): consumes a 2-tuple of equal-length arrays (Table 1)."""

    def __repr__(self) -> str:
        return "zip"


@dataclass(frozen=True)
class ZipWith(Expr):
    """zip(env[name], input): the partial application dot(x) of Fig. 5 zips a
    captured vector with each row.  Not a pattern of the paper."""

    name: str

    def __repr__(self) -> str:
        return f"zip({self.name}, _)"


@dataclass(frozen=True)
class Split(Expr):
    n: int

    def __repr__(self) -> str:
        return f"split-{self.n}"


@dataclass(frozen=True)
class Join(Expr):
    def __repr__(self) -> str:
        return "join"


@dataclass(frozen=True)
class Iterate(Expr):
    n: int
    f: Any

    def __repr__(self) -> str:
        return f"iterate-{self.n}({self.f!r})"


@dataclass(frozen=True)
class Reorder(Expr):
    def __repr__(self) -> str:
        return "reorder"


@dataclass(frozen=True)
class ReorderStride(Expr):
    """reorder-stride^s; give s, or n with n * s = len (then s = len / n)."""

    s: Optional[int] = None
    n: Optional[int] = None

    def __repr__(self) -> str:
        if self.s is not None:
            return f"reorder-stride-{self.s}"
        if self.n is not None:
            return f"reorder-stride(n={self.n})"
        return "reorder-stride"


@dataclass(frozen=True)
class ToLocal(Expr):
    f: Any

    def __repr__(self) -> str:
        return f"toLocal({self.f!r})"


@dataclass(frozen=True)
class ToGlobal(Expr):
    f: Any

    def __repr__(self) -> str:
        return f"toGlobal({self.f!r})"


@dataclass(frozen=True)
class AsVector(Expr):
    n: int

    def __repr__(self) -> str:
        return f"asVector-{self.n}"


@dataclass(frozen=True)
class AsScalar(Expr):
    def __repr__(self) -> str:
        return "asScalar"


@dataclass(frozen=True)
class Vect(Expr):
    """vect^n(f): f vectorised by n (Table 2).  Appears where a user
    function may appear."""

    n: int
    f: Any

    def __repr__(self) -> str:
        return f"vectorize-{self.n}({self.f!r})"


@dataclass(frozen=True)
class Id(Expr):
    def __repr__(self) -> str:
        return "id"


@dataclass(frozen=True)
class PadTo(Expr):
    """Append copies of z until the outer dimension has length L.  Not a
    pattern of the paper: it states the neutral-element padding a kernel
    applies to a ragged tail (z = 0 is neutral for add, and abs(0) = 0,
    0 * y = 0 keep the padded elements neutral after the map)."""

    L: int
    z: Any = 0

    def __repr__(self) -> str:
        return f"pad-{self.L}"


def C(*fs) -> Any:
    """Composition helper: C(f, g, h) = f . g . h; nested Composes are
    flattened and a single function is returned unchanged."""
    flat = []
    for f in fs:
        if isinstance(f, Compose):
            flat.extend(f.fs)
        else:
            flat.append(f)
    if len(flat) == 1:
        return flat[0]
    return Compose(tuple(flat))


def is_function(f) -> bool:
    """User functions (and their vectorised forms) act on primitives."""
    return isinstance(f, (UserFun, Vect))


# ============================================================================
# Types
# ============================================================================
@dataclass(frozen=True)
class ArrT:
    """T[d0][d1]...; ``vw`` > 1 means the element is a vector Tvw;
    ``pair`` marks an array of pairs <T,T> (zip); ``space`` is the address
    space of the storage (toLocal/toGlobal)."""

    dims: Tuple[int, ...]
    vw: int = 1
    pair: bool = False
    space: str = "global"

    def with_dims(self, dims, **kw) -> "ArrT":
        d = dict(dims=tuple(dims), vw=self.vw, pair=self.pair, space=self.space)
        d.update(kw)
        return ArrT(**d)


@dataclass(frozen=True)
class TupT:
    items: Tuple[ArrT, ...]


PARALLEL = ("map-workgroup", "map-local", "map-global")


def _check_nesting(kind: str, ctx: Tuple[str, ...]) -> None:
    """Sec. 4.2 "Maps": the OpenCL thread hierarchy must be respected."""
    inside_par = [k for k in ctx if k in PARALLEL]
    inside_seq = "seq" in ctx
    if kind in PARALLEL and inside_seq:
        raise PatternTypeError(f"{kind} nested inside a sequential pattern")
    if kind == "map-workgroup" and inside_par:
        raise PatternTypeError("map-workgroup nested inside another parallel map")
    if kind == "map-global" and inside_par:
        raise PatternTypeError("map-global nested inside another parallel map")
    if kind == "map-local":
        if "map-workgroup" not in ctx:
            raise PatternTypeError("map-local outside a map-workgroup")
        if "map-local" in ctx or "map-global" in ctx:
            raise PatternTypeError("map-local nested inside map-local/map-global")


def _fun_type(f, t: ArrT) -> ArrT:
    """Type of a user function applied to one element of type t (dims == ())."""
    if isinstance(f, Vect):
        if t.vw != f.n:
            raise PatternTypeError(f"vectorize-{f.n} applied to elements of width {t.vw}")
        _fun_type(f.f, ArrT((), 1, t.pair, t.space))
        return ArrT((), t.vw, False, t.space)
    if t.vw != 1:
        raise PatternTypeError(f"scalar function {f!r} applied to a vector element")
    a = arity(f)
    if f.name == "fold":
        raise PatternTypeError("a reduction function cannot be mapped")
    if a == 2 and not t.pair:
        raise PatternTypeError(f"binary function {f!r} mapped over non-pairs")
    if a == 1 and t.pair:
        raise PatternTypeError(f"unary function {f!r} mapped over pairs")
    return ArrT((), 1, False, t.space)


def infer(e, t, ctx: Tuple[str, ...] = ()):
    """Output type of expression ``e`` applied to a value of type ``t``."""
    if isinstance(e, Compose):
        for f in reversed(e.fs):
            t = infer(f, t, ctx)
        return t
    if isinstance(e, Zip):
        if not isinstance(t, TupT) or len(t.items) != 2:
            raise PatternTypeError("zip expects two arrays")
        a, b = t.items
        if a.dims[:1] != b.dims[:1] or len(a.dims) != 1 or len(b.dims) != 1:
            raise PatternTypeError(f"zip of arrays of lengths {a.dims} and {b.dims}")
        if a.vw != 1 or b.vw != 1 or a.pair or b.pair:
            raise PatternTypeError("zip of non-scalar arrays")
        return ArrT(a.dims, 1, True, a.space)
    if isinstance(t, TupT):
        raise PatternTypeError(f"{e!r} applied to a tuple of arrays (zip first)")
    if isinstance(e, ZipWith):
        if len(t.dims) != 1 or t.pair or t.vw != 1:
            raise PatternTypeError("zip with a captured vector needs a flat scalar array")
        return t.with_dims(t.dims, pair=True)
    if isinstance(e, Map):
        _check_nesting(e.kind, ctx)
        if len(t.dims) < 1:
            raise PatternTypeError(f"{e.kind} applied to a primitive")
        inner = t.with_dims(t.dims[1:])
        if is_function(e.f):
            if inner.dims != ():
                raise PatternTypeError(f"user function {e.f!r} mapped over arrays {inner.dims}")
            out = _fun_type(e.f, inner)
        else:
            sub = ctx + ((e.kind,) if e.kind != "map-seq" else ("map-seq", "seq"))
            out = infer(e.f, inner, sub)
        return out.with_dims((t.dims[0],) + out.dims)
    if isinstance(e, Reduce):
        if len(t.dims) != 1:
            raise PatternTypeError(f"{e.kind} needs a one-dimensional input, got {t.dims}")
        _reduce_fun_check(e.f, t)
        return t.with_dims((1,), pair=False)
    if isinstance(e, Split):
        if e.n < 1 or len(t.dims) < 1 or t.dims[0] % e.n != 0:
            raise PatternTypeError(f"split-{e.n} of an outer dimension {t.dims[:1]}")
        return t.with_dims((t.dims[0] // e.n, e.n) + t.dims[1:])
    if isinstance(e, Join):
        if len(t.dims) < 2:
            raise PatternTypeError("join needs at least two dimensions")
        return t.with_dims((t.dims[0] * t.dims[1],) + t.dims[2:])
    if isinstance(e, Iterate):
        if e.n < 0:
            raise PatternTypeError("iterate with a negative count")
        for _ in range(e.n):
            t = infer(e.f, t, ctx)
        return t
    if isinstance(e, (Reorder, Id)):
        return t
    if isinstance(e, ReorderStride):
        if len(t.dims) < 1:
            raise PatternTypeError("reorder-stride of a primitive")
        _stride_params(e, t.dims[0])
        return t
    if isinstance(e, ToLocal):
        return infer(e.f, t, ctx).with_dims(infer(e.f, t, ctx).dims, space="local")
    if isinstance(e, ToGlobal):
        return infer(e.f, t, ctx).with_dims(infer(e.f, t, ctx).dims, space="global")
    if isinstance(e, AsVector):
        if t.vw != 1 or len(t.dims) < 1 or t.dims[-1] % e.n != 0 or e.n < 2:
            raise PatternTypeError(f"asVector-{e.n} of {t.dims} (width {t.vw})")
        return t.with_dims(t.dims[:-1] + (t.dims[-1] // e.n,), vw=e.n)
    if isinstance(e, AsScalar):
        if t.vw == 1 or len(t.dims) < 1:
            raise PatternTypeError("asScalar of a scalar array")
        return t.with_dims(t.dims[:-1] + (t.dims[-1] * t.vw,), vw=1)
    if isinstance(e, PadTo):
        if len(t.dims) < 1 or e.L < t.dims[0]:
            raise PatternTypeError(f"pad-{e.L} of {t.dims}")
        return t.with_dims((e.L,) + t.dims[1:])
    raise PatternTypeError(f"cannot type {e!r}")


def _reduce_fun_check(f, t: ArrT) -> None:
    base = f.f if isinstance(f, Vect) else f
    if isinstance(f, Vect) and f.n != t.vw:
        raise PatternTypeError(f"vectorize-{f.n} reduction over width-{t.vw} elements")
    if not isinstance(f, Vect) and t.vw != 1:
        raise PatternTypeError("scalar reduction function over vector elements")
    if base.name == "fold":
        g = base.params[1]
        if arity(g) == 2 and not t.pair:
            raise PatternTypeError("fused reduction of a binary function over non-pairs")
        if arity(g) == 1 and t.pair:
            raise PatternTypeError("fused reduction of a unary function over pairs")
    else:
        if arity(base) != 2:
            raise PatternTypeError(f"reduction with non-binary {base!r}")
        if t.pair:
            raise PatternTypeError("plain reduction over pairs")


def _stride_params(e: ReorderStride, L: int) -> Tuple[int, int]:
    if e.s is not None:
        s = e.s
        if s < 1 or L % s != 0:
            raise PatternTypeError(f"reorder-stride-{s} of length {L}")
        return s, L // s
    if e.n is not None:
        n = e.n
        if n < 1 or L % n != 0:
            raise PatternTypeError(f"reorder-stride(n={n}) of length {L}")
        return L // n, n
    raise PatternTypeError("reorder-stride without a stride: lower it first")


# ============================================================================
# Values
# ============================================================================
@dataclass
class Arr:
    """Array value: ``data`` holds batch axes, then the logical dimensions,
    then a lane axis when vw > 1."""

    data: np.ndarray
    vw: int = 1


@dataclass
class Pair:
    """Array of pairs (zip): two component arrays of identical layout."""

    a: np.ndarray
    b: np.ndarray
    vw: int = 1


@dataclass
class Tup:
    items: Tuple[Arr, ...]


def _both(v, fn):
    if isinstance(v, Pair):
        return Pair(fn(v.a), fn(v.b), v.vw)
    return Arr(fn(v.data), v.vw)


def _ndim_logical(v, nb: int) -> int:
    d = v.a if isinstance(v, Pair) else v.data
    return d.ndim - nb - (1 if v.vw > 1 else 0)


# ---------------------------------------------------------------------------
# arithmetic of user functions
# ---------------------------------------------------------------------------
class _Arith:
    def __init__(self, mode: str):
        if mode not in ("f64", "f32", "int"):
            raise ValueError(mode)
        self.mode = mode
        self.dtype = {"f64": np.float64, "f32": np.float32, "int": np.int64}[mode]

    def cast_in(self, x):
        return np.asarray(x, dtype=self.dtype)

    def const(self, c):
        return self.dtype(c)

    def apply(self, f, *args):
        """Apply user function ``f`` elementwise (lanes included)."""
        if isinstance(f, Vect):
            return self.apply(f.f, *args)
        n = f.name
        if n == "abs":
            (x,) = args
            return np.where(x < 0, -x, x)  # Fig. 5: if (x < 0) -x else x
        if n == "id":
            return args[0]
        if n == "neg":
            return -args[0]
        if n == "add":
            return args[0] + args[1]
        if n == "add64":
            r = np.asarray(args[0], np.float64) + np.asarray(args[1], np.float64)
            return r
        if n == "mult":
            return args[0] * args[1]
        if n == "square":
            return args[0] * args[0]
        if n == "sqrt64":
            return np.sqrt(np.asarray(args[0], np.float64))
        if n == "mul3":
            return args[0] * self.const(3)
        if n == "mult_by":
            a = f.params[0]
            x = args[0]
            return np.asarray(x.dtype.type(a) * x) if self.mode != "int" else a * x
        if n == "to_f32":
            return np.asarray(args[0]).astype(np.float32).astype(self.dtype)
        if n == "to_f64":
            return np.asarray(args[0], np.float64)
        if n == "compose":
            g_out = self.apply(f.params[1], *args)
            return self.apply(f.params[0], g_out)
        if n == "fold":
            acc, x = args
            fh, fg = f.params
            gx = self.apply(fg, *x) if isinstance(x, tuple) else self.apply(fg, x)
            return self.apply(fh, acc, gx)
        raise PatternTypeError(f"unknown user function {n}")


_UFUNC = {"add": np.add, "add64": np.add, "mult": np.multiply}

FOLD_CHUNK = 1 << 20


def _fold_axis(ar: _Arith, f, z, v, ax: int):
    """Left fold of ``v`` along axis ``ax``: acc = z; acc = f(acc, e_i) in
    order.  For f = h(acc, g(x)) with h one of add/mult, g(x) does not depend
    on acc, so it is evaluated for every element first and the fold is then
    ufunc.accumulate, which numpy evaluates strictly in sequence (the same
    operations, in the same order, as the loop).  Other functions fall back
    to an explicit Python loop."""
    base = f.f if isinstance(f, Vect) else f
    if base.name == "fold":
        h, g = base.params
        if isinstance(v, Pair):
            pre = ar.apply(g, v.a, v.b)
        else:
            pre = ar.apply(g, v.data)
    else:
        h = base
        if isinstance(v, Pair):
            raise PatternTypeError("plain reduction over pairs")
        pre = v.data
    pre = np.asarray(pre)
    if h.name == "add64":
        pre = pre.astype(np.float64)
        dt = np.float64
    else:
        dt = pre.dtype
    shape = list(pre.shape)
    m = shape[ax]
    del shape[ax]
    acc = np.full(shape, z, dtype=dt) if np.isscalar(z) else np.broadcast_to(
        np.asarray(z, dtype=dt), shape).copy()
    uf = _UFUNC.get(h.name)
    if uf is None:
        for i in range(m):
            acc = ar.apply(h, acc, np.take(pre, i, axis=ax))
        return acc
    for c0 in range(0, m, FOLD_CHUNK):
        chunk = np.take(pre, np.arange(c0, min(m, c0 + FOLD_CHUNK)), axis=ax)
        block = np.concatenate([np.expand_dims(acc, ax), chunk.astype(dt, copy=False)], axis=ax)
        acc = np.take(uf.accumulate(block, axis=ax, dtype=dt), -1, axis=ax)
    return acc


def _comp_fold_axis(v, ax: int):
    """Neumaier-compensated left fold of ``v`` along axis ``ax`` (see
    ReduceSeqComp), every operation in the mode's arithmetic (numpy float32
    arithmetic rounds each operation to nearest, as the kernels' explicit
    fp32 operations do)."""
    if isinstance(v, Pair):
        raise PatternTypeError("compensated reduction over pairs")
    d = np.asarray(v.data)
    shape = list(d.shape)
    m = shape[ax]
    del shape[ax]
    s = np.zeros(shape, dtype=d.dtype)
    c = np.zeros(shape, dtype=d.dtype)
    with np.errstate(invalid="ignore", over="ignore"):
        for i in range(m):
            t = np.take(d, i, axis=ax)
            u = s + t
            big = np.abs(s) >= np.abs(t)
            c = c + np.where(big, (s - u) + t, (t - u) + s)
            s = u
        if d.dtype.kind == "f":
            return np.where(np.isfinite(s), s + c, s)
    return s + c


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------
def _eval(e, v, nb: int, ar: _Arith, env: Dict[str, np.ndarray]):
    if isinstance(e, Compose):
        for f in reversed(e.fs):
            v = _eval(f, v, nb, ar, env)
        return v
    if isinstance(e, Zip):
        a, b = v.items
        return Pair(a.data, b.data, 1)
    if isinstance(e, ZipWith):
        cap = env[e.name]
        if cap.shape != v.data.shape[nb:]:
            raise PatternTypeError(f"zip of {e.name}{cap.shape} with rows {v.data.shape[nb:]}")
        return Pair(np.broadcast_to(cap, v.data.shape), v.data, 1)
    if isinstance(e, Map):
        if is_function(e.f):
            if isinstance(v, Pair):
                return Arr(np.asarray(ar.apply(e.f, v.a, v.b)), v.vw)
            return Arr(np.asarray(ar.apply(e.f, v.data)), v.vw)
        return _eval(e.f, v, nb + 1, ar, env)
    if isinstance(e, Reduce):
        if e.kind == "reduce-seq-comp":
            acc = _comp_fold_axis(v, nb)
        else:
            acc = _fold_axis(ar, e.f, e.z, v, nb)
        return Arr(np.expand_dims(np.asarray(acc), nb), v.vw)
    if isinstance(e, Split):
        def sp(d):
            m = d.shape[nb]
            return d.reshape(d.shape[:nb] + (m // e.n, e.n) + d.shape[nb + 1:])
        return _both(v, sp)
    if isinstance(e, Join):
        def jn(d):
            return d.reshape(d.shape[:nb] + (d.shape[nb] * d.shape[nb + 1],) + d.shape[nb + 2:])
        return _both(v, jn)
    if isinstance(e, Iterate):
        for _ in range(e.n):
            v = _eval(e.f, v, nb, ar, env)
        return v
    if isinstance(e, (Reorder, Id)):
        return v
    if isinstance(e, ReorderStride):
        d0 = v.a if isinstance(v, Pair) else v.data
        L = d0.shape[nb]
        s, n = _stride_params(e, L)
        i = np.arange(L)
        idx = i // n + s * (i % n)   # Sec. 3.2: out[i] = in[i/n + s*(i mod n)]
        return _both(v, lambda d: np.take(d, idx, axis=nb))
    if isinstance(e, (ToLocal, ToGlobal)):
        return _eval(e.f, v, nb, ar, env)
    if isinstance(e, AsVector):
        def av(d):
            m = d.shape[-1]
            return d.reshape(d.shape[:-1] + (m // e.n, e.n))
        out = _both(v, av)
        out.vw = e.n
        return out
    if isinstance(e, AsScalar):
        def asc(d):
            return d.reshape(d.shape[:-2] + (d.shape[-2] * d.shape[-1],))
        out = _both(v, asc)
        out.vw = 1
        return out
    if isinstance(e, PadTo):
        def pd(d):
            m = d.shape[nb]
            if e.L == m:
                return d
            pad_shape = d.shape[:nb] + (e.L - m,) + d.shape[nb + 1:]
            return np.concatenate([d, np.full(pad_shape, e.z, dtype=d.dtype)], axis=nb)
        return _both(v, pd)
    raise PatternTypeError(f"cannot evaluate {e!r}")


def type_of(x) -> Union[ArrT, TupT]:
    if isinstance(x, tuple):
        return TupT(tuple(type_of(i) for i in x))
    a = np.asarray(x)
    return ArrT(tuple(a.shape))


def evaluate(e, x, mode: str = "f64", env: Optional[Dict[str, np.ndarray]] = None):
    """Type-check ``e`` against the input and evaluate it.

    ``x`` is one array or a tuple of arrays (the inputs of a zip).  In mode
    'f32' every input must be exactly representable in fp32.  Returns a
    numpy array with the output's logical shape (plus a lane axis if the
    output elements are vectors)."""
    env = dict(env or {})
    t = type_of(x)
    infer(e, t)
    ar = _Arith(mode)

    def conv(a):
        a = np.asarray(a)
        if mode == "f32":
            a32 = a.astype(np.float32)
            if not np.array_equal(a32.astype(a.dtype), a, equal_nan=True):
                raise ValueError("input not exactly representable in fp32")
            return a32
        return ar.cast_in(a)

    if isinstance(x, tuple):
        v = Tup(tuple(Arr(conv(i)) for i in x))
    else:
        v = Arr(conv(x))
    env = {k: conv(val) for k, val in env.items()}
    out = _eval(e, v, 0, ar, env)
    if isinstance(out, Pair):
        return (out.a, out.b)
    return out.data
