"""Autotuner: time every kernel variant of an op over a set of shapes.

The paper chooses its split sizes and vector widths "by exploring different
values empirically" (Sec. 6.2); this module does that exploration on the
device.  For each (op, shape) it launches every variant through the C-ABI
and times it with CUDA events on the launching stream: a CUDA graph of R
back-to-back calls (R disjoint input slices when the working set is below
twice the L2 size, so every call reads cold data from HBM; R = 1 otherwise)
is replayed ``reps`` times and the median replay time divided by R is the
per-call time.  One JSON record per (device, op, shape, variant) is appended
to a database file.  Records
already present are skipped, so an interrupted sweep resumes where it
stopped.  ``write_table`` turns a database into the nearest-shape table the
TABLE policy of the library reads.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import lift

L2_BYTES = 129 * 1000 * 1000
MIXED = (lift.OP_ASUM_BF16, lift.OP_DOT_BF16, lift.OP_ASUM_FP8, lift.OP_DOT_FP8)


def op_bytes(op: int, n: int, M: int = 0, N: int = 0) -> int:
    """Algorithmic bytes one call moves."""
    if op in (lift.OP_ASUM, lift.OP_NRM2, lift.OP_SUM, lift.OP_ASUM_COMP):
        return 4 * n
    if op == lift.OP_DOT_COMP:
        return 8 * n
    if op in (lift.OP_AXPY, lift.OP_BLACKSCHOLES):
        return 12 * n
    if op == lift.OP_DOT:
        return 8 * n
    if op == lift.OP_SCAL:
        return 8 * n
    if op == lift.OP_GEMV:
        return 4 * M * N + 4 * N + 8 * M
    if op == lift.OP_GEMV_T:
        return 4 * M * N + 4 * M + 8 * N
    elem = 2 if op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16) else 1
    scales = 4 * math.ceil(n / 4096) if op in (lift.OP_ASUM_FP8, lift.OP_DOT_FP8) else 0
    k = 2 if op in (lift.OP_DOT_BF16, lift.OP_DOT_FP8) else 1
    return k * (elem * n + scales)


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


POOL_BYTES = 1 << 30   # rotation pool: every call of a small shape reads cold data
MAX_ROT = 64


def rotation(nbytes: int) -> int:
    """Calls in one timed graph: for working sets of at least twice the L2
    (cold anyway) as many slices of the 1 GiB pool as fit, up to 4 (so the
    event resolution is shared by several calls), else enough distinct
    slices that a slice is evicted before it is read again."""
    if nbytes >= 2 * L2_BYTES:
        return int(max(1, min(4, POOL_BYTES // max(nbytes, 1))))
    return int(max(2, min(MAX_ROT, POOL_BYTES // max(nbytes, 1))))


class Pools:
    """1 GiB device arrays (random contents) that every shape slices; the
    R slices of a call rotation sit POOL_BYTES / R apart, so the R calls of
    a small shape together touch more than the L2 holds."""

    def __init__(self, seed: int = 0):
        import torch
        self.torch = torch
        self.g = torch.Generator(device="cuda")
        self.g.manual_seed(seed)
        self.cache = {}

    def get(self, name: str, kind: str):
        if name not in self.cache:
            t, g = self.torch, self.g
            if kind == "f32":
                a = t.randn(POOL_BYTES // 4, device="cuda", generator=g)
            elif kind == "bf16":
                a = t.randn(POOL_BYTES // 2, device="cuda", generator=g).to(t.bfloat16)
            elif kind == "price":   # stock prices U(5, 30)
                a = t.rand(POOL_BYTES // 4, device="cuda", generator=g) * 25.0 + 5.0
            elif kind == "u8":   # E4M3 codes below 0x7E: finite values, no NaN
                a = t.randint(0, 0x7E, (POOL_BYTES,), device="cuda", generator=g, dtype=t.uint8)
            else:                # block scales
                a = t.rand(1 << 20, device="cuda", generator=g) + 0.5
            self.cache[name] = a
        return self.cache[name]


class Buffers:
    """Slices of the pools for one shape: R disjoint, evenly spread slices
    of each array (timing does not depend on the values)."""

    def __init__(self, pools: Pools, op: int, n: int, M: int, N: int):
        self.op, self.n, self.M, self.N = op, n, M, N
        self.R = rotation(op_bytes(op, n, M, N))
        self.pools = pools
        self.res = pools.torch.zeros(self.R * 64, device="cuda")

    def _slice(self, name, kind, r, count):
        a = self.pools.get(name, kind)
        stride = (a.numel() // self.R) // 256 * 256
        assert count <= stride or self.R == 1, "slice larger than its share of the pool"
        assert count <= a.numel()
        return a[r * stride: r * stride + count]

    def call(self, vid: int, r: int):
        """The r-th call of the rotation for variant vid."""
        op, n, M, N = self.op, self.n, self.M, self.N
        res = self.res[64 * r:64 * r + 1]
        if op in (lift.OP_ASUM, lift.OP_NRM2, lift.OP_SUM):
            x = self._slice("x", "f32", r, n)
            fn = {lift.OP_ASUM: lift.lift_asum_v, lift.OP_NRM2: lift.lift_nrm2_v,
                  lift.OP_SUM: lift.lift_sum_v}[op]
            return lambda: fn(vid, x, n, res)
        if op == lift.OP_AXPY:
            x, y = self._slice("x", "f32", r, n), self._slice("y", "f32", r, n)
            return lambda: lift.lift_axpy_v(vid, n, 1.5, x, y)
        if op == lift.OP_ASUM_COMP:
            x = self._slice("x", "f32", r, n)
            return lambda: lift.lift_asum_comp_v(vid, x, n, res)
        if op == lift.OP_DOT_COMP:
            x, y = self._slice("x", "f32", r, n), self._slice("y", "f32", r, n)
            return lambda: lift.lift_dot_comp_v(vid, x, y, n, res)
        if op == lift.OP_DOT:
            x, y = self._slice("x", "f32", r, n), self._slice("y", "f32", r, n)
            return lambda: lift.lift_dot_v(vid, x, y, n, res)
        if op == lift.OP_SCAL:
            x, y = self._slice("x", "f32", r, n), self._slice("y", "f32", r, n)
            return lambda: lift.lift_scal_v(vid, n, 1.5, x, y)
        if op == lift.OP_BLACKSCHOLES:
            sp = self._slice("price", "price", r, n)
            c, p = self._slice("y", "f32", r, n), self._slice("x", "f32", r, n)
            return lambda: lift.lift_blackscholes_v(vid, n, sp, 20.0, 0.02, 0.3, 1.0, c, p)
        if op == lift.OP_GEMV_T:
            A = self._slice("x", "f32", r, M * N)
            y = self._slice("y", "f32", r, N)
            xv = self._slice("gx", "f32", 0, M)
            return lambda: lift.lift_gemv_t_v(vid, M, N, 1.0, A, N, xv, 0.5, y)
        if op == lift.OP_GEMV:
            A = self._slice("x", "f32", r, M * N)
            y = self._slice("y", "f32", r, M)
            xv = self._slice("gx", "f32", 0, N)
            return lambda: lift.lift_gemv_v(vid, M, N, 1.0, A, N, xv, 0.5, y)
        bf = op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16)
        dt = lift.BF16 if bf else lift.FP8_E4M3
        kind = "bf16" if bf else "u8"
        x, y = self._slice("x" + kind, kind, r, n), self._slice("y" + kind, kind, r, n)
        nb = max(1, math.ceil(n / 4096))
        xs = None if bf else self.pools.get("xs", "scale")[:nb]
        ys = None if bf else self.pools.get("ys", "scale")[:nb]
        if op in (lift.OP_ASUM_BF16, lift.OP_ASUM_FP8):
            return lambda: lift.lift_asum_ex_v(vid, dt, x, xs, n, res)
        return lambda: lift.lift_dot_ex_v(vid, dt, x, xs, y, ys, n, res)


class Timer:
    """Time R calls captured in one CUDA graph; a replay runs the calls back
    to back on one stream, so the host's launch overhead and the event
    resolution do not enter the per-call time."""

    def __init__(self):
        import torch
        self.torch = torch

    def per_call_ms(self, calls, reps: int, warmup: int) -> float:
        torch = self.torch
        for _ in range(warmup):
            for c in calls:
                c()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for c in calls:
                c()
        g.replay()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(s)
            g.replay()
            b.record(s)
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ev) / len(calls)
        del g
        return ms


def _key(rec) -> Tuple:
    return (rec["device"], rec["op"], rec["n"], rec["M"], rec["N"], rec["variant"])


def load_db(path: str) -> List[Dict]:
    if not path or not os.path.exists(path):
        return []
    out = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line:
                out.append(json.loads(line))
    return out


def sweep(shapes: Iterable[Tuple[int, int, int, int]], db_path: Optional[str], reps: int = 20,
          warmup: int = 2, variants: Optional[Dict[int, List[int]]] = None,
          verbose: bool = False) -> List[Dict]:
    """Time every variant of each (op, n, M, N); returns the new records."""
    import torch
    lift.lift_init()
    dkey = device_key()
    done = {_key(r) for r in load_db(db_path)} if db_path else set()
    timer = Timer()
    pools = Pools()
    out = []
    f = open(db_path, "a") if db_path else None
    t_start, n_shapes = time.perf_counter(), 0
    try:
        for (op, n, M, N) in shapes:
            vids = variants.get(op) if variants else None
            vids = vids if vids is not None else list(range(lift.lift_variant_count(op)))
            todo = [v for v in vids if (dkey, op, n, M, N, v) not in done]
            if not todo:
                continue
            buf = Buffers(pools, op, n, M, N)
            nbytes = op_bytes(op, n, M, N)
            for v in todo:
                ms = timer.per_call_ms([buf.call(v, r) for r in range(buf.R)], reps, warmup)
                rec = {"device": dkey, "op": op, "opname": lift.OP_NAMES[op], "n": n, "M": M,
                       "N": N, "variant": v, "name": lift.lift_variant_describe(op, v)["name"],
                       "ms": ms, "bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
                       "reps": reps, "rotation": buf.R}
                out.append(rec)
                if f:
                    f.write(json.dumps(rec) + "\n")
            if f:
                f.flush()
            if verbose:
                best = min((r for r in out if (r["op"], r["n"], r["M"], r["N"]) == (op, n, M, N)),
                           key=lambda r: r["ms"])
                print(f"{lift.OP_NAMES[op]:10s} n={n} M={M} N={N}: best {best['name']} "
                      f"{best['ms'] * 1e3:.1f} us {best['gbs']:.0f} GB/s", flush=True)
            del buf
            n_shapes += 1
    finally:
        if f:
            f.close()
    if verbose and out:
        wall = time.perf_counter() - t_start
        print(f"swept {n_shapes} shapes, {len(out)} timings in {wall:.1f} s "
              f"({wall / max(1, n_shapes):.2f} s per shape)", flush=True)
    assert lift.lift_read_status() == 0, "a kernel reported a device-side timeout"
    return out


CSV_HEADER = "device,op,n,M,N,variant,ms"


def export_csv(records: List[Dict], path: str) -> None:
    """Compact copy of a timing database (one line per measurement)."""
    with open(path, "w") as f:
        f.write(CSV_HEADER + "\n")
        for r in records:
            f.write(f"{r['device']},{r['op']},{r['n']},{r['M']},{r['N']},{r['variant']},{r['ms']:.6g}\n")


def load_csv(path: str) -> List[Dict]:
    out = []
    with open(path) as f:
        head = f.readline().strip()
        assert head == CSV_HEADER, head
        for line in f:
            d, op, n, M, N, v, ms = line.strip().split(",")
            out.append({"device": d, "op": int(op), "n": int(n), "M": int(M), "N": int(N),
                        "variant": int(v), "ms": float(ms)})
    return out


def best_per_shape(records: List[Dict]) -> Dict[Tuple, Dict]:
    best: Dict[Tuple, Dict] = {}
    for r in records:
        k = (r["op"], r["n"], r["M"], r["N"])
        if k not in best or r["ms"] < best[k]["ms"]:
            best[k] = r
    return best


def write_table(records: List[Dict], path: str) -> None:
    """Nearest-shape table: 'op log2(n+1) log2(M+1) log2(N+1) variant'."""
    with open(path, "w") as f:
        f.write("# op log2(n+1) log2(M+1) log2(N+1) variant  (best measured variant)\n")
        for (op, n, M, N), r in sorted(best_per_shape(records).items()):
            nn = M * N if op == lift.OP_GEMV else n
            f.write(f"{op} {math.log2(nn + 1):.6f} {math.log2(M + 1):.6f} {math.log2(N + 1):.6f} "
                    f"{r['variant']}\n")


# ---------------------------------------------------------------------------
# shape sets
# ---------------------------------------------------------------------------
def workload_shapes() -> List[Tuple[int, int, int, int]]:
    """The benchmark configurations: asum 2^20, dot / scal / asum 2^26, the
    two gemv shapes, the mixed ops at 2^28, nrm2 / sum / axpy 2^26, the two
    gemv-T shapes, BlackScholes at 2^22 (the paper's size) and 2^26, the
    compensated asum / dot at 2^26."""
    s = [(lift.OP_ASUM, 1 << 20, 0, 0), (lift.OP_DOT, 1 << 26, 0, 0), (lift.OP_SCAL, 1 << 26, 0, 0),
         (lift.OP_ASUM, 1 << 26, 0, 0),
         (lift.OP_GEMV, 8192 * 8192, 8192, 8192), (lift.OP_GEMV, 65536 * 1024, 65536, 1024)]
    s += [(op, 1 << 28, 0, 0) for op in MIXED]
    s += [(op, 1 << 26, 0, 0) for op in (lift.OP_NRM2, lift.OP_SUM, lift.OP_AXPY)]
    s += [(lift.OP_GEMV_T, 8192 * 8192, 8192, 8192), (lift.OP_GEMV_T, 65536 * 1024, 65536, 1024)]
    s += [(lift.OP_BLACKSCHOLES, 1 << 22, 0, 0), (lift.OP_BLACKSCHOLES, 1 << 26, 0, 0)]
    s += [(lift.OP_ASUM_COMP, 1 << 26, 0, 0), (lift.OP_DOT_COMP, 1 << 26, 0, 0)]
    return s


# op ids of the first training distribution (asum, dot, scal, gemv and the
# four mixed-precision ops); the others are drawn by passing ``ops``
DEFAULT_SHAPE_OPS = tuple(range(8))


def random_shapes(count: int, seed: int, ops: Optional[List[int]] = None,
                  lo: int = 8, hi: int = 28,
                  gemv_range: Tuple[float, float] = (6, 14),
                  align_n: int = 1) -> List[Tuple[int, int, int, int]]:
    """Shapes for the cost model: op uniform over ``ops``; vector lengths
    round(2^U(lo, hi)); gemv M, N = round(2^U(gemv_range)) (N rounded up to
    a multiple of ``align_n``) with 2^8 <= M*N <= 2^28."""
    rng = np.random.default_rng(seed)
    ops = ops or list(DEFAULT_SHAPE_OPS)
    out = []
    while len(out) < count:
        op = int(rng.choice(ops))
        if op in (lift.OP_GEMV, lift.OP_GEMV_T):
            M = int(round(2 ** rng.uniform(*gemv_range)))
            N = int(round(2 ** rng.uniform(*gemv_range)))
            N = -(-N // align_n) * align_n
            if M * N > (1 << 28) or M * N < (1 << 8):
                continue
            out.append((op, M * N, M, N))
        else:
            out.append((op, int(round(2 ** rng.uniform(lo, hi))), 0, 0))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--db", required=True)
    ap.add_argument("--preset", default="workloads", choices=["workloads", "train", "heldout"])
    ap.add_argument("--count", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--table", default=None)
    ap.add_argument("--csv", default=None)
    ap.add_argument("--ops", type=int, nargs="+", default=None,
                    help="restrict to these op codes")
    ap.add_argument("--gemv-range", type=float, nargs=2, default=(6, 14),
                    help="log2 range of gemv M and N for random shapes")
    ap.add_argument("--align-n", type=int, default=1,
                    help="round random gemv N up to a multiple of this")
    ap.add_argument("--derived", action="store_true",
                    help="time only the variants a rule derivation reaches (derive.py)")
    ap.add_argument("--variant-names", nargs="+", default=None,
                    help="time only variants whose names start with one of these")
    ap.add_argument("--shapes-from", default=None,
                    help="time the shapes of an existing timing CSV (filtered by --ops)")
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    if a.shapes_from:
        shapes = sorted({(r["op"], r["n"], r["M"], r["N"]) for r in load_csv(a.shapes_from)
                         if a.ops is None or r["op"] in a.ops})
    elif a.preset == "workloads":
        shapes = [s for s in workload_shapes() if a.ops is None or s[0] in a.ops]
    else:
        shapes = random_shapes(a.count, a.seed, a.ops, gemv_range=tuple(a.gemv_range),
                               align_n=a.align_n)
    variants = None
    if a.derived or a.variant_names:
        from . import derive
        variants = {}
        for op in sorted({sh[0] for sh in shapes}):
            ids = list(range(lift.lift_variant_count(op)))
            if a.derived:
                name = next((k for k, v in derive.OP_IDS.items() if v == op), None)
                if name is not None:
                    ids = derive.derivable_variants(name)
            if a.variant_names:
                ids = [v for v in ids if lift.lift_variant_describe(op, v)["name"].startswith(
                    tuple(a.variant_names))]
            variants[op] = ids
    sweep(shapes, a.db, reps=a.reps, variants=variants, verbose=a.v)
    if a.table:
        write_table(load_db(a.db), a.table)
    if a.csv:
        export_csv(load_db(a.db), a.csv)


if __name__ == "__main__":
    main()
