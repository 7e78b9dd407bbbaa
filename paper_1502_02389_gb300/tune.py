"""Autotuner: time every kernel variant of an op over a set of shapes.

The paper chooses its split sizes and vector widths "by exploring different
values empirically" (Sec. 6.2); this module does that exploration on the
device.  For each (op, shape) it launches every variant through the C-ABI,
times it with CUDA events on the launching stream (median of ``reps`` after
``warmup`` calls; the L2 is flushed by reading a 512 MiB buffer before each
timed call when the working set is below twice the L2 size), and appends one
JSON record per (device, op, shape, variant) to a database file.  Records
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
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import lift

L2_BYTES = 129 * 1000 * 1000
MIXED = (lift.OP_ASUM_BF16, lift.OP_DOT_BF16, lift.OP_ASUM_FP8, lift.OP_DOT_FP8)


def op_bytes(op: int, n: int, M: int = 0, N: int = 0) -> int:
    """Algorithmic bytes one call moves."""
    if op == lift.OP_ASUM:
        return 4 * n
    if op == lift.OP_DOT:
        return 8 * n
    if op == lift.OP_SCAL:
        return 8 * n
    if op == lift.OP_GEMV:
        return 4 * M * N + 4 * N + 8 * M
    elem = 2 if op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16) else 1
    scales = 4 * math.ceil(n / 4096) if op in (lift.OP_ASUM_FP8, lift.OP_DOT_FP8) else 0
    k = 2 if op in (lift.OP_DOT_BF16, lift.OP_DOT_FP8) else 1
    return k * (elem * n + scales)


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


class Buffers:
    """Device inputs of one shape (random contents; timing does not depend
    on the values)."""

    def __init__(self, op: int, n: int, M: int, N: int, seed: int = 0):
        import torch
        g = torch.Generator(device="cuda")
        g.manual_seed(seed)
        self.op, self.n, self.M, self.N = op, n, M, N
        dev = "cuda"
        self.r = torch.zeros(1, device=dev)
        if op in (lift.OP_ASUM, lift.OP_DOT, lift.OP_SCAL):
            self.x = torch.randn(max(n, 1), device=dev, generator=g)
            self.y = torch.randn(max(n, 1), device=dev, generator=g) if op != lift.OP_ASUM else None
        elif op == lift.OP_GEMV:
            self.A = torch.randn(max(M * N, 1), device=dev, generator=g)
            self.x = torch.randn(max(N, 1), device=dev, generator=g)
            self.y = torch.randn(max(M, 1), device=dev, generator=g)
        else:
            nbytes = n * (2 if op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16) else 1)
            # bf16: draw N(0,1) values and keep their bf16 bits; fp8: bytes
            # below 0x7F / 0xFF avoid the NaN codes
            if op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16):
                self.x = torch.randn(max(n, 1), device=dev, generator=g).to(torch.bfloat16)
                self.y = torch.randn(max(n, 1), device=dev, generator=g).to(torch.bfloat16)
            else:
                self.x = torch.randint(0, 0x7E, (max(nbytes, 1),), device=dev, generator=g,
                                       dtype=torch.uint8)
                self.y = torch.randint(0, 0x7E, (max(nbytes, 1),), device=dev, generator=g,
                                       dtype=torch.uint8)
            nb = max(1, math.ceil(n / 4096))
            self.xs = torch.rand(nb, device=dev, generator=g) + 0.5
            self.ys = torch.rand(nb, device=dev, generator=g) + 0.5

    def call(self, vid: int):
        op, n = self.op, self.n
        if op == lift.OP_ASUM:
            return lambda: lift.lift_asum_v(vid, self.x, n, self.r)
        if op == lift.OP_DOT:
            return lambda: lift.lift_dot_v(vid, self.x, self.y, n, self.r)
        if op == lift.OP_SCAL:
            return lambda: lift.lift_scal_v(vid, n, 1.5, self.x, self.y)
        if op == lift.OP_GEMV:
            return lambda: lift.lift_gemv_v(vid, self.M, self.N, 1.0, self.A, self.N, self.x, 0.5,
                                            self.y)
        dt = lift.BF16 if op in (lift.OP_ASUM_BF16, lift.OP_DOT_BF16) else lift.FP8_E4M3
        xs = self.xs if dt == lift.FP8_E4M3 else None
        ys = self.ys if dt == lift.FP8_E4M3 else None
        if op in (lift.OP_ASUM_BF16, lift.OP_ASUM_FP8):
            return lambda: lift.lift_asum_ex_v(vid, dt, self.x, xs, n, self.r)
        return lambda: lift.lift_dot_ex_v(vid, dt, self.x, xs, self.y, ys, n, self.r)


class Timer:
    def __init__(self):
        import torch
        self.torch = torch
        self.flush_buf = torch.ones(128 << 20, device="cuda")   # 512 MiB

    def median_ms(self, fn, reps: int, warmup: int, flush: bool) -> float:
        torch = self.torch
        for _ in range(warmup):
            fn()
        s = torch.cuda.current_stream()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            if flush:
                self.flush_buf.sum()
            a.record(s)
            fn()
            b.record(s)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)


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


def sweep(shapes: Iterable[Tuple[int, int, int, int]], db_path: Optional[str], reps: int = 10,
          warmup: int = 2, variants: Optional[Dict[int, List[int]]] = None,
          verbose: bool = False) -> List[Dict]:
    """Time every variant of each (op, n, M, N); returns the new records."""
    import torch
    lift.lift_init()
    dkey = device_key()
    done = {_key(r) for r in load_db(db_path)} if db_path else set()
    timer = Timer()
    out = []
    f = open(db_path, "a") if db_path else None
    try:
        for (op, n, M, N) in shapes:
            vids = variants.get(op) if variants else None
            vids = vids if vids is not None else list(range(lift.lift_variant_count(op)))
            todo = [v for v in vids if (dkey, op, n, M, N, v) not in done]
            if not todo:
                continue
            buf = Buffers(op, n, M, N)
            nbytes = op_bytes(op, n, M, N)
            flush = nbytes < 2 * L2_BYTES
            for v in todo:
                ms = timer.median_ms(buf.call(v), reps, warmup, flush)
                rec = {"device": dkey, "op": op, "opname": lift.OP_NAMES[op], "n": n, "M": M,
                       "N": N, "variant": v, "name": lift.lift_variant_describe(op, v)["name"],
                       "ms": ms, "bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
                       "reps": reps, "flushed": flush}
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
            torch.cuda.empty_cache()
    finally:
        if f:
            f.close()
    assert lift.lift_read_status() == 0, "a kernel reported a device-side timeout"
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
    """The benchmark configurations (asum 2^20, dot/scal 2^26, the two gemv
    shapes, the mixed ops at 2^28)."""
    s = [(lift.OP_ASUM, 1 << 20, 0, 0), (lift.OP_DOT, 1 << 26, 0, 0), (lift.OP_SCAL, 1 << 26, 0, 0),
         (lift.OP_ASUM, 1 << 26, 0, 0),
         (lift.OP_GEMV, 8192 * 8192, 8192, 8192), (lift.OP_GEMV, 65536 * 1024, 65536, 1024)]
    s += [(op, 1 << 28, 0, 0) for op in MIXED]
    return s


def random_shapes(count: int, seed: int, ops: Optional[List[int]] = None,
                  lo: int = 8, hi: int = 28) -> List[Tuple[int, int, int, int]]:
    """Shapes for the cost model: op uniform over ``ops``; vector lengths
    round(2^U(lo, hi)); gemv M, N = round(2^U(6, 14)) with M*N <= 2^28."""
    rng = np.random.default_rng(seed)
    ops = ops or list(range(lift.NUM_OPS))
    out = []
    while len(out) < count:
        op = int(rng.choice(ops))
        if op == lift.OP_GEMV:
            M = int(round(2 ** rng.uniform(6, 14)))
            N = int(round(2 ** rng.uniform(6, 14)))
            if M * N > (1 << 28):
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
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--table", default=None)
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    if a.preset == "workloads":
        shapes = workload_shapes()
    else:
        shapes = random_shapes(a.count, a.seed)
    sweep(shapes, a.db, reps=a.reps, verbose=a.v)
    if a.table:
        write_table(load_db(a.db), a.table)


if __name__ == "__main__":
    main()
