"""Rewrite rules of arXiv 1502.02389, Sec. 4 (Fig. 3 algorithmic rules,
Fig. 4 OpenCL-specific lowering rules), as tree rewrites.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

A rule either rewrites one node (``node rules``) or two adjacent functions
of a composition ``a . b`` (``pair rules``; ``b`` is applied first).  A rule
raises ``NotApplicable`` when its left-hand side does not match.
``rewrite(e, path, rule, **params)`` applies a rule at a position: ``path``
is a tuple of steps, an int selecting an item of a ``Compose`` and ``'f'``
selecting the function argument of map/reduce/iterate/toLocal/toGlobal/vect.
For a pair rule the path ends at the ``Compose`` and ``at=i`` names the pair
(fs[i], fs[i+1]).

Each rule states one equation, so the value of an expression does not change
under any rule (Sec. 4.3: derivations are "semantically equivalent by
construction"); the tests check exactly that with the interpreter.
"""
from __future__ import annotations

import dataclasses
from typing import Any, Callable, Dict, List, Optional, Tuple

from .patterns import (AsScalar, AsVector, ArrT, C, Compose, Id, Iterate, Join,
                       Map, PatternTypeError, Reduce, Reorder, ReorderStride,
                       Split, ToGlobal, ToLocal, TupT, UserFun, Vect, compose_fun,
                       fold, infer, is_function)


class NotApplicable(Exception):
    """The rule's left-hand side does not match here."""


# ============================================================================
# Fig. 3a -- iterate decomposition: iterate^(m+n)(f) -> iterate^m(f) . iterate^n(f)
# ============================================================================
def iterate_decomposition(e, m: int, t=None):
    if not isinstance(e, Iterate) or not (0 <= m <= e.n):
        raise NotApplicable
    return C(Iterate(m, e.f), Iterate(e.n - m, e.f))


# ============================================================================
# Fig. 3b -- reorder commutativity
#   map(f) . reorder -> reorder . map(f);   reorder . map(f) -> map(f) . reorder
# ============================================================================
def reorder_commutativity(a, b, t=None):
    if isinstance(a, Map) and a.kind == "map" and isinstance(b, Reorder):
        return C(b, a)
    if isinstance(a, Reorder) and isinstance(b, Map) and b.kind == "map":
        return C(b, a)
    raise NotApplicable


# ============================================================================
# Fig. 3c -- split-join: map(f) -> join . map(map(f)) . split^n
# ============================================================================
def split_join(e, n: int, t=None):
    if not isinstance(e, Map) or e.kind != "map":
        raise NotApplicable
    return C(Join(), Map(Map(e.f)), Split(n))


# ============================================================================
# Fig. 3d -- reduction and partial reduction
#   reduce(f,z)   -> reduce(f,z) . part-red(f,z)
#   part-red(f,z) -> reduce(f,z)
#                  | part-red(f,z) . reorder
#                  | join . map(part-red(f,z)) . split^n
#                  | iterate^n(part-red(f,z))
# ============================================================================
def _is(e, kind):
    return isinstance(e, Reduce) and e.kind == kind


def reduction(e, t=None):
    if not _is(e, "reduce"):
        raise NotApplicable
    return C(Reduce(e.f, e.z), Reduce(e.f, e.z, "part-red"))


def partred_to_reduce(e, t=None):
    if not _is(e, "part-red"):
        raise NotApplicable
    return Reduce(e.f, e.z)


def partred_reorder(e, t=None):
    if not _is(e, "part-red"):
        raise NotApplicable
    return C(e, Reorder())


def partred_split(e, n: int, t=None):
    if not _is(e, "part-red"):
        raise NotApplicable
    return C(Join(), Map(e), Split(n))


def partred_iterate(e, n: int, t=None):
    if not _is(e, "part-red"):
        raise NotApplicable
    return Iterate(n, e)


# ============================================================================
# Fig. 3e -- simplification: split^n . join^n | join^n . split^n -> id,
#            asVector^n . asScalar^n | asScalar^n . asVector^n -> id
# ============================================================================
def simplify_split_join(a, b, t=None):
    """split^n . join^n -> id: ``t`` is the input type of the pair (the
    join's input); its inner dimension must be n."""
    if isinstance(a, Split) and isinstance(b, Join):
        if t is None or not isinstance(t, ArrT) or len(t.dims) < 2 or t.dims[1] != a.n:
            raise NotApplicable
        return Id()
    raise NotApplicable


def simplify_join_split(a, b, t=None):
    if isinstance(a, Join) and isinstance(b, Split):
        return Id()
    raise NotApplicable


def simplify_vector(a, b, t=None):
    if isinstance(a, AsVector) and isinstance(b, AsScalar):
        if t is None or not isinstance(t, ArrT) or t.vw != a.n:
            raise NotApplicable
        return Id()
    if isinstance(a, AsScalar) and isinstance(b, AsVector):
        return Id()
    raise NotApplicable


def drop_id(a, b, t=None):
    """f . id -> f and id . f -> f (definition of id; used to tidy up after
    the simplification rules)."""
    if isinstance(b, Id):
        return a
    if isinstance(a, Id):
        return b
    raise NotApplicable


# ============================================================================
# Fig. 3f -- fusion
#   map(f) . map(g) -> map(f . g)
#   reduce-seq(f,z) . map-seq(g) -> reduce-seq(lambda acc,x: f(acc, g(x)), z)
# ============================================================================
def fuse_maps(a, b, t=None):
    if isinstance(a, Map) and isinstance(b, Map) and a.kind == b.kind:
        if is_function(a.f) and is_function(b.f):
            if isinstance(a.f, Vect) or isinstance(b.f, Vect):
                raise NotApplicable
            return Map(compose_fun(a.f, b.f), a.kind)
        if is_function(a.f) != is_function(b.f):
            raise NotApplicable
        return Map(C(a.f, b.f), a.kind)
    raise NotApplicable


def fuse_reduce_seq(a, b, t=None):
    if _is(a, "reduce-seq") and isinstance(b, Map) and b.kind == "map-seq":
        if not is_function(a.f) or not is_function(b.f):
            raise NotApplicable
        if isinstance(a.f, Vect) or isinstance(b.f, Vect):
            if not (isinstance(a.f, Vect) and isinstance(b.f, Vect) and a.f.n == b.f.n):
                raise NotApplicable
            return Reduce(Vect(a.f.n, fold(a.f.f, b.f.f)), a.z, "reduce-seq")
        if a.f.name == "fold":
            raise NotApplicable
        return Reduce(fold(a.f, b.f), a.z, "reduce-seq")
    raise NotApplicable


# ============================================================================
# Fig. 4a -- map -> map-workgroup | map-local | map-global | map-seq
# Fig. 4b -- reduce -> reduce-seq (the only lowering)
# Fig. 4c -- reorder -> reorder-stride^s | id
# Fig. 4d -- map-local(f) -> toGlobal(map-local(f)) | toLocal(map-local(f))
# Fig. 4e -- map(f) -> asScalar . map(vect^n(f)) . asVector^n  (once per map)
# ============================================================================
def lower_map(e, kind: str, t=None):
    if not isinstance(e, Map) or e.kind != "map":
        raise NotApplicable
    if kind not in ("map-workgroup", "map-local", "map-global", "map-seq"):
        raise NotApplicable
    return Map(e.f, kind)


def lower_reduce(e, t=None):
    if not _is(e, "reduce"):
        raise NotApplicable
    return Reduce(e.f, e.z, "reduce-seq")


def lower_reorder(e, s: Optional[int] = None, n: Optional[int] = None, t=None):
    if not isinstance(e, Reorder):
        raise NotApplicable
    if s is None and n is None:
        return Id()
    return ReorderStride(s=s, n=n)


def to_global(e, t=None):
    if not isinstance(e, Map) or e.kind != "map-local":
        raise NotApplicable
    return ToGlobal(e)


def to_local(e, t=None):
    if not isinstance(e, Map) or e.kind != "map-local":
        raise NotApplicable
    return ToLocal(e)


def vectorize(e, n: int, t=None):
    """Sec. 4.2 "Vectorization": applicable once to a map; the check is the
    function's type -- a function that is already vectorised is refused."""
    if not isinstance(e, Map) or e.kind != "map" or not is_function(e.f):
        raise NotApplicable
    if isinstance(e.f, Vect):
        raise NotApplicable
    return C(AsScalar(), Map(Vect(n, e.f)), AsVector(n))


NODE_RULES: Dict[str, Callable] = {
    "iterate_decomposition": iterate_decomposition,
    "split_join": split_join,
    "reduction": reduction,
    "partred_to_reduce": partred_to_reduce,
    "partred_reorder": partred_reorder,
    "partred_split": partred_split,
    "partred_iterate": partred_iterate,
    "lower_map": lower_map,
    "lower_reduce": lower_reduce,
    "lower_reorder": lower_reorder,
    "to_global": to_global,
    "to_local": to_local,
    "vectorize": vectorize,
}

PAIR_RULES: Dict[str, Callable] = {
    "reorder_commutativity": reorder_commutativity,
    "simplify_split_join": simplify_split_join,
    "simplify_join_split": simplify_join_split,
    "simplify_vector": simplify_vector,
    "fuse_maps": fuse_maps,
    "fuse_reduce_seq": fuse_reduce_seq,
    "drop_id": drop_id,
}


# ============================================================================
# Engine
# ============================================================================
def _child(e, step):
    if isinstance(step, int):
        if not isinstance(e, Compose):
            raise KeyError(step)
        return e.fs[step]
    if step == "f":
        return e.f
    raise KeyError(step)


def _replace(e, path, new):
    if not path:
        return new
    step, rest = path[0], path[1:]
    if isinstance(step, int):
        fs = list(e.fs)
        fs[step] = _replace(fs[step], rest, new)
        return C(*fs)
    return dataclasses.replace(e, f=_replace(e.f, rest, new))


def input_type_at(e, path, t):
    """Type of the value that reaches the node at ``path`` when ``e`` is
    applied to a value of type ``t`` (None where the node is a user
    function rather than an array pattern)."""
    for step in path:
        if isinstance(step, int):
            for f in reversed(e.fs[step + 1:]):
                t = infer(f, t)
            e = e.fs[step]
        else:
            if isinstance(e, Map):
                t = t.with_dims(t.dims[1:])
            elif isinstance(e, (ToLocal, ToGlobal, Iterate)):
                pass
            else:
                t = None
            e = e.f
    return t


def rewrite(e, path, rule: str, t=None, at: Optional[int] = None, **params):
    """Apply rule ``rule`` at ``path`` of ``e``.  ``t`` is the input type of
    ``e``; it is needed by the rules whose side condition is a size."""
    node = e
    for step in path:
        node = _child(node, step)
    if rule in NODE_RULES:
        sub_t = input_type_at(e, path, t) if t is not None else None
        new = NODE_RULES[rule](node, t=sub_t, **params)
        return _replace(e, tuple(path), new)
    if rule in PAIR_RULES:
        if not isinstance(node, Compose) or at is None or at + 1 >= len(node.fs):
            raise NotApplicable
        sub_t = None
        if t is not None:
            sub_t = input_type_at(e, tuple(path) + (at + 1,), t)
        new = PAIR_RULES[rule](node.fs[at], node.fs[at + 1], t=sub_t, **params)
        fs = list(node.fs[:at]) + [new] + list(node.fs[at + 2:])
        return _replace(e, tuple(path), C(*fs))
    raise KeyError(rule)


def positions(e, path=()):
    """All node paths of ``e`` (array patterns and nested functions)."""
    out = [tuple(path)]
    if isinstance(e, Compose):
        for i, f in enumerate(e.fs):
            out += positions(f, tuple(path) + (i,))
    elif isinstance(e, (Map, Iterate, ToLocal, ToGlobal)) and not is_function(e):
        if not isinstance(e.f, UserFun):
            out += positions(e.f, tuple(path) + ("f",))
    return out


def well_typed(e, t) -> bool:
    try:
        infer(e, t)
        return True
    except PatternTypeError:
        return False
