"""Low-level expressions: the ones the paper prints (Fig. 2b, Fig. 8, Fig. 9)
and the parametrised expression each GPU kernel variant evaluates.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The kernel-variant expressions are written only with the patterns of
Table 1 and Table 2 (plus ``PadTo`` for the neutral padding of a ragged
tail).  Evaluated in the interpreter's fp32 mode they state, operation by
operation, the arithmetic of an fp32 kernel whose CTAs are workgroups and
whose threads are local threads: per-thread sequential folds
(reduce-seq), lane-wise vectors (asVector / vect), coalescing order
(reorder-stride), halving trees (iterate over split-2), and an FP64 final
combine.  A kernel built from the same expression must agree bit for bit.
"""
from __future__ import annotations

import math

from .patterns import (AsScalar, AsVector, C, Id, Iterate, Join, Map, MapLocal, MapSeq,
                       MapWorkgroup, PadTo, PartRed, Reduce, ReduceSeq, ReduceSeqComp, Reorder,
                       ReorderStride, Split, ToGlobal, ToLocal, Vect, Zip, ZipWith, abs_,
                       absAndPlus, add, add64, fold, id_, mul3, mult, mult_by, sqrt64, square,
                       to_f32, to_f64)

# the fused reduction function of each reduce program (rule 3f applied to
# reduce(add, 0) . map(g)); sum has no map and folds add itself
FOLD = {"asum": absAndPlus, "dot": fold(add, mult), "nrm2": fold(add, square), "sum": add}


# ============================================================================
# Fig. 2b -- vectorScal = join . map-workgroup(asScalar . map-local(
#            vectorize-4(mul3)) . asVector-4) . split-1024
# ============================================================================
def fig2b_vector_scal():
    return C(Join(),
             MapWorkgroup(C(AsScalar(), MapLocal(Vect(4, mul3)), AsVector(4))),
             Split(1024))


# ============================================================================
# Fig. 8 -- the fused asum derivation, equations (1) to (8), as printed
# (eq. (8) closes the parenthesis the figure leaves open)
# ============================================================================
def fig8_equations(n: int):
    PR = PartRed(add, 0)
    R = Reduce(add, 0)
    return [
        C(R, Map(abs_)),                                                    # (1)
        C(R, Join(), Map(PR), Split(n), Map(abs_)),                         # (2)
        C(R, Join(), Map(PR), Split(n), Join(), Map(Map(abs_)), Split(n)),  # (3)
        C(R, Join(), Map(PR), Map(Map(abs_)), Split(n)),                    # (4)
        C(R, Join(), Map(C(PR, Map(abs_))), Split(n)),                      # (5)
        C(R, Join(), Map(C(PR, MapSeq(abs_))), Split(n)),                   # (6)
        C(R, Join(), Map(C(ReduceSeq(add, 0), MapSeq(abs_))), Split(n)),    # (7)
        C(R, Join(), Map(ReduceSeq(absAndPlus, 0)), Split(n)),              # (8)
    ]


# ============================================================================
# Fig. 9 -- device-specific asum expressions.  Fig. 9 writes reorder-stride
# without its stride; it is read as s = len / n_next, n_next being the size
# of the split that follows (s = 128 in (a), s = 256 in (b)).  The outer
# reduce-seq carries no arguments in the figure; they are (add, 0).
# "absAnd+" in (c) is absAndPlus.
# ============================================================================
def fig9a_nvidia():
    return C(
        ReduceSeq(add, 0), Join(),
        MapWorkgroup(C(
            Join(), ToGlobal(MapLocal(MapSeq(id_))), Split(1),
            Iterate(7, C(Join(), MapLocal(ReduceSeq(add, 0)), Split(2))),
            Join(), ToLocal(MapLocal(ReduceSeq(absAndPlus, 0))), Split(2048),
            ReorderStride(n=2048))),
        Split(262144))


def fig9b_amd():
    v4 = lambda f: Vect(4, f)  # noqa: E731
    return C(
        ReduceSeq(add, 0), Join(), AsScalar(),
        MapWorkgroup(C(
            Join(), ToGlobal(MapLocal(MapSeq(v4(id_)))), Split(1),
            Iterate(8, C(Join(), MapLocal(ReduceSeq(v4(add), 0)), Split(2))),
            Join(), ToLocal(MapLocal(ReduceSeq(v4(absAndPlus), 0))), Split(2),
            ReorderStride(n=2))),
        AsVector(4), Split(2048))


def fig9c_intel():
    return C(
        ReduceSeq(add, 0), Join(), AsScalar(),
        MapWorkgroup(C(
            Join(), MapLocal(ReduceSeq(Vect(4, absAndPlus), 0)), Split(8192))),
        AsVector(4), Split(32768))


# ============================================================================
# Kernel variants
# ============================================================================
WARP = 32


def halving_tree(plus=add):
    """One warp-wide halving tree: iterate-5(join . map-local(reduce-seq(+))
    . split-2 . reorder-stride(n=2)).  Each level pairs element j with
    element j + len/2, which is what a shuffle-down by len/2 computes."""
    level = C(Join(), MapLocal(ReduceSeq(plus, 0)), Split(2), ReorderStride(n=2))
    return Iterate(5, level)


def block_tree(threads: int, plus=add):
    """[threads] -> [1]: a halving tree inside every warp, then the warp
    results (padded with zeros to one warp) through one more warp tree."""
    warps = threads // WARP
    e = C(Join(), Map(halving_tree(plus)), Split(WARP))
    if warps > 1:
        e = C(halving_tree(plus), PadTo(WARP), e)
    return e


def _thread_order(threads: int, per_thread: int, J: int, stride: bool):
    """Vectors of one CTA (its tiles in order, J per thread per tile) ->
    [threads][per_thread]; thread t takes, tile by tile, vectors
    t + threads*j (stride) or t*J + j (contiguous chunk)."""
    if stride:
        return C(Split(per_thread), ReorderStride(s=threads))
    return C(Split(per_thread), Join(), ReorderStride(s=threads), Split(J))


def final_combine(P: int, ft: int, cast32: bool = True, post=None):
    """[P] fp32 partials -> [1]: thread t of one CTA of ft threads sums
    partials t, t+ft, ... in FP64, then an FP64 block tree; ``post`` (a user
    function such as sqrt64) is mapped over the FP64 sum; the result is
    rounded to fp32 when cast32."""
    M = max(1, math.ceil(P / ft))
    body = C(block_tree(ft, add64), Join(),
             MapLocal(ReduceSeq(add64, 0)), Split(M), ReorderStride(s=ft),
             PadTo(ft * M), Map(to_f64))
    if post is not None:
        body = C(Map(post), body)
    if cast32:
        body = C(Map(to_f32), body)
    return C(Join(), MapWorkgroup(body), Split(P))


def cta_expr(op: str, K: int, tile: int, vw: int, threads: int, stride: bool = True):
    """One CTA folding K tiles of ``tile`` elements (in order) into one
    value: every thread folds its J vectors of each tile from zero (over
    vect^vw lanes) and adds the tile's lanes in order, adds its K tile
    values with the compensated reduce-seq (the partial reduction of Fig. 3d
    applied to the thread's reduce-seq, its outer level compensated), then
    the block tree."""
    V = tile // vw
    J = V // threads
    assert V % threads == 0 and tile % vw == 0
    f = FOLD[op]
    fr = Vect(vw, f) if vw > 1 else f
    tile_value = ReduceSeq(fr, 0)
    if vw > 1:          # the tile's lane sums added in order
        tile_value = C(ReduceSeq(add, 0), AsScalar(), ReduceSeq(fr, 0))
    per_thread = C(ReduceSeqComp(add), Join(), Map(tile_value), Split(J))
    return C(block_tree(threads), Join(), MapLocal(per_thread),
             _thread_order(threads, K * J, J, stride),
             AsVector(vw) if vw > 1 else Id())


def batch_reduce(op: str, n: int, item: int, tile: int, vw: int, threads: int = 256,
                 ft: int = 256, cast32: bool = True):
    """One asum/dot op of the batched launch: split^item into work items,
    each folded by one CTA like a kernel tile sequence (cta_expr), then
    the FP64 combine of the item partials in item order."""
    P = max(1, math.ceil(n / item))
    K = item // tile
    L = P * item
    e = C(final_combine(P, ft, cast32), Join(), MapWorkgroup(cta_expr(op, K, tile, vw, threads)),
          Split(item), PadTo(L))
    if op == "dot":
        e = C(e, Zip())
    return e, L


def reduce_variant(op: str, n: int, tile: int, vw: int, threads: int, grid: int,
                   stride: bool = True, cluster: int = 1, ft: int = 256,
                   cast32: bool = True):
    """Expression of a fp32 asum/dot kernel variant and the padded input
    length it expects (the input padded with zeros to that length).

    Tiles of ``tile`` elements go to the ``grid`` CTAs round robin
    (CTA b takes tiles b, b+grid, ...: reorder-stride^grid at tile level);
    every thread folds its vectors in order into ``vw`` lane accumulators
    (reduce-seq over vect^vw(absAndPlus) or of the fused multiply-add
    fold), adds its lanes in order, then the CTA runs ``block_tree``; with a
    cluster, ``cluster`` consecutive CTA results are added in rank order;
    the partials are combined by ``final_combine``."""
    if op not in FOLD:
        raise ValueError(op)
    T = max(1, math.ceil(n / tile))
    K = math.ceil(T / grid)
    L = grid * K * tile
    V = tile // vw
    J = V // threads
    assert V % threads == 0 and tile % vw == 0 and grid % cluster == 0
    cta = cta_expr(op, K, tile, vw, threads, stride)
    parts = C(Join(), MapWorkgroup(cta), Split(K * tile), Join(),
              ReorderStride(s=grid), Split(tile), PadTo(L))
    P = grid
    if cluster > 1:
        parts = C(Join(), Map(ReduceSeq(add, 0)), Split(cluster), parts)
        P = grid // cluster
    e = C(final_combine(P, ft, cast32, sqrt64 if op == "nrm2" else None), parts)
    if op == "dot":
        e = C(e, Zip())
    return e, L


GEMV_GROUP = 8   # vectors a gemv lane folds plainly before a compensated add


def grouped_dot(vw: int, J: int, group: int = GEMV_GROUP):
    """[J] zipped vectors of one lane -> [1]: groups of ``group``
    consecutive vectors (the last padded with zeros), each folded from zero
    over the vw lanes with its lanes then added in order, and the group
    values added with the compensated reduce-seq (the partial reduction of
    Fig. 3d applied to the lane's reduce-seq, its outer level
    compensated)."""
    f = fold(add, mult)
    fr = Vect(vw, f) if vw > 1 else f
    value = ReduceSeq(fr, 0)
    if vw > 1:
        value = C(ReduceSeq(add, 0), AsScalar(), ReduceSeq(fr, 0))
    Jp = max(group, math.ceil(J / group) * group)
    return C(ReduceSeqComp(add), Join(), Map(value), Split(group), PadTo(Jp))


def gemv_row_variant(N: int, vw: int, lanes: int = WARP):
    """Expression of one row of the gemv kernel: ``lanes`` threads share the
    row; lane l takes vectors l, l+lanes, ... of the zero-padded row
    (zipped with x) in order and folds them with ``grouped_dot``, then
    ``block_tree``."""
    chunk = lanes * vw
    Np = max(chunk, math.ceil(N / chunk) * chunk)
    J = Np // chunk
    return C(block_tree(lanes), Join(), MapLocal(grouped_dot(vw, J)),
             Split(J), ReorderStride(s=lanes),
             AsVector(vw) if vw > 1 else Id(), PadTo(Np), ZipWith("x"))


def gemv_z_variant(M: int, N: int, alpha, vw: int, lanes: int = WARP,
                   rows_per_cta: int = 1):
    """z = alpha * (row dots), rows grouped rows_per_cta to a CTA."""
    assert M % rows_per_cta == 0
    row = gemv_row_variant(N, vw, lanes)
    return C(Map(mult_by(alpha)), Join(), Join(),
             MapWorkgroup(Map(row)), Split(rows_per_cta))


def gemv_split_z_variant(M: int, N: int, alpha, vw: int, threads: int, L: int, S: int):
    """z of the split-row gemv: each row zipped with x, padded to S*L and
    split into S segments of L elements; a CTA of ``threads`` folds a
    segment (thread t takes vectors t, t+threads, ... in order and folds
    them with ``grouped_dot``, then ``block_tree``); the S segment partials
    of the row are added by one warp (lane l adds partials l, l+32, ...
    with the compensated reduce-seq, then a halving tree) and multiplied by
    alpha -- the partial-reduction rule of Fig. 3 applied to each row's
    reduce."""
    chunk = threads * vw
    assert L % chunk == 0 and S * L >= N
    J = L // chunk
    segment = C(block_tree(threads), Join(), MapLocal(grouped_dot(vw, J)),
                Split(J), ReorderStride(s=threads), AsVector(vw) if vw > 1 else Id())
    per = max(1, math.ceil(S / WARP))
    lanes = C(halving_tree(add), Join(), MapLocal(ReduceSeqComp(add)), Split(per),
              ReorderStride(s=WARP), PadTo(WARP * per))
    row = C(Join(), MapWorkgroup(lanes), Split(S), Join(), MapWorkgroup(segment), Split(L),
            PadTo(S * L), ZipWith("x"))
    return C(Map(mult_by(alpha)), Join(), Map(row))


def gemv_t_z_variant(M: int, N: int, alpha, B: int, RB: int, passes: int = 1,
                     cluster: int = 1, group: int = 32):
    """z of the gemv-T kernel: every column of A (the rows of the
    reorder-stride view) zipped with x, padded to RB*B, folded in RB blocks
    of B rows (fp32; a block's rows in groups of ``group``, each group
    folded from zero, the group sums added with the compensated reduce-seq);
    the block partials are then combined in fp32 --
    one pass: added in block order with the compensated reduce-seq; one pass
    with clusters of ``cluster`` blocks: each cluster's consecutive block
    partials added in order, then the cluster sums added in order with the
    compensated reduce-seq (the partial reduction of Fig. 3d applied to the
    block partials); two pass: lane l of one warp adds partials l, l+32,
    ..., then a halving tree over the lanes -- and multiplied by alpha."""
    if passes == 1 and cluster > 1:
        assert RB % cluster == 0
        combine = C(ReduceSeqComp(add), Join(), Map(ReduceSeq(add, 0)), Split(cluster))
    elif passes == 1:
        combine = ReduceSeqComp(add)
    else:
        per = max(1, math.ceil(RB / WARP))
        lanes = C(halving_tree(add), Join(), MapLocal(ReduceSeqComp(add)), Split(per),
                  ReorderStride(s=WARP), PadTo(WARP * per))
        combine = C(Join(), MapWorkgroup(lanes), Split(RB))     # one warp per column
    Bp = math.ceil(B / group) * group
    block = C(ReduceSeqComp(add), Join(), Map(ReduceSeq(fold(add, mult), 0)), Split(group),
              PadTo(Bp))
    col = C(combine, Join(), Map(block), Split(B), PadTo(RB * B), ZipWith("x"))
    return C(Map(mult_by(alpha)), Join(), Map(col), Split(M), ReorderStride(s=N), Join())
