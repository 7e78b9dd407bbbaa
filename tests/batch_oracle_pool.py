"""Checking every op of a large batch against the oracle on all host cores.

Test infrastructure (imported by the GPU tests only).  The batch's operands
live in one device pool; the pool is read back in contiguous groups of ops
(about ``chunk_bytes`` each) into one of two shared-memory buffers, and
spawned worker processes -- one per host core -- evaluate each op of the
group with the oracle while the next group is read back into the other
buffer.  A worker returns, per op, its largest |got - oracle| / tolerance.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

ASUM, DOT, GEMV = 0, 1, 3   # op ids of the batched workload

_ATTACHED = {}


def _view(name: str, count: int):
    shm = _ATTACHED.get(name)
    if shm is None:
        shm = _ATTACHED[name] = shared_memory.SharedMemory(name=name)
    return np.ndarray((count,), np.float32, buffer=shm.buf)


def _check(task):
    """task: (shared-memory name, elements in it, [(op index, op, offsets
    relative to the buffer, initial gemv output or None), ...])."""
    from oracle import blas
    name, count, items = task
    buf = _view(name, count)
    out = []
    for i, d, e, y0 in items:
        get = lambda k, c: buf[e[k]:e[k] + c].astype(np.float64)  # noqa: E731
        if d["op"] == GEMV:
            M, N = d["M"], d["N"]
            A, x = get("A", M * N).reshape(M, N), get("x", N)
            ref = blas.gemv(A, x, y0.astype(np.float64), 1.0, 0.5)
            tol = blas.tolerance(N, 1.0) * blas.gemv_row_terms(A, x, y0, 1.0, 0.5)
            r = np.abs(get("out", M) - ref) / tol
            out.append((i, float(np.max(r)) if r.size else 0.0))
        else:
            x = get("x", d["n"])
            if d["op"] == ASUM:
                ref, terms = blas.asum(x), blas.asum_terms(x)
            else:
                y = get("y", d["n"])
                ref, terms = blas.dot(x, y), blas.dot_terms(x, y)
            got = float(buf[e["out"]])
            tol = blas.tolerance(d["n"], terms)
            out.append((i, abs(got - ref) / tol if tol > 0 else float(got != ref)))
    return out


def _span(d, e):
    """First and one-past-last pool element of an op's arrays."""
    ends = [e["out"] + (d["M"] if d["op"] == GEMV else 1)]
    for k, c in (("A", d["M"] * d["N"]), ("x", d["N"] if d["op"] == GEMV else d["n"]),
                 ("y", d["n"])):
        if k in e:
            ends.append(e[k] + c)
    return min(e.values()), max(ends)


def _groups(ops, lay, chunk_elems: int):
    """Consecutive ops whose arrays span at most chunk_elems pool elements
    (the layout places each op's arrays after the previous op's)."""
    def span(i):
        return _span(ops[i], lay[i])

    group, lo, hi = [], None, None
    for i in range(len(ops)):
        a, b = span(i)
        if group and b - lo > chunk_elems:
            yield group, lo, hi
            group, lo = [], None
        if lo is None:
            lo = a
        hi = b
        group.append(i)
    if group:
        yield group, lo, hi


def check_all(pool, ops, lay, y0, chunk_bytes: int = 1 << 30):
    """Every op of the batch against the oracle.  pool: the torch device
    tensor holding the batch's arrays after one run; y0: {op index: initial
    gemv output (numpy)}.  Returns {op index: ratio} and the worker count."""
    import torch
    procs = max(1, len(os.sched_getaffinity(0)))
    try:
        st = os.statvfs("/dev/shm")
        chunk_bytes = int(min(chunk_bytes, st.f_bavail * st.f_frsize // 3))
    except OSError:
        pass
    widest = max(b - a for a, b in (_span(d, e) for d, e in zip(ops, lay)))
    chunk_elems = max(chunk_bytes // 4, widest)     # every op fits in one group
    bufs = [shared_memory.SharedMemory(create=True, size=chunk_elems * 4) for _ in range(2)]
    ratios = {}
    views = None
    try:
        views = [torch.from_numpy(np.ndarray((chunk_elems,), np.float32, buffer=b.buf))
                 for b in bufs]
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as workers:
            pending = [None, None]
            for g, (idx, lo, hi) in enumerate(_groups(ops, lay, chunk_elems)):
                k = g % 2
                if pending[k] is not None:          # the buffer's previous group is done
                    for i, r in pending[k].get():
                        ratios[i] = r
                views[k][:hi - lo].copy_(pool[lo:hi])
                items = [(i, ops[i], {key: off - lo for key, off in lay[i].items()},
                          y0.get(i)) for i in idx]
                per = max(1, len(items) // (4 * procs))
                tasks = [(bufs[k].name, chunk_elems, items[j:j + per])
                         for j in range(0, len(items), per)]
                pending[k] = _Joined(workers.map_async(_check, tasks))
            for p in pending:
                if p is not None:
                    for i, r in p.get():
                        ratios[i] = r
    finally:
        views = None          # drop the exported views before closing the buffers
        for b in bufs:
            try:
                b.close()
            except BufferError:
                pass
            b.unlink()
    return ratios, procs


class _Joined:
    """map_async result flattened to one list of (op index, ratio)."""

    def __init__(self, res):
        self.res = res

    def get(self):
        return [t for part in self.res.get() for t in part]
