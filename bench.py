"""Benchmark of the liftblas hot path on GB300.

Default workload (the dot/scal configuration): fp32 vectors x, y of
n = 2^26 elements ~ N(0,1) (seed 1), alpha = 1.5.  One step is
dot(x, y) and scal(alpha, x) -> z with the variants the cost model picks,
submitted through the C-ABI as two calls (``--mode calls``, the default)
or as one batched persistent launch (``--mode batched``); the other
submission is measured too and reported in ``config``, with the learned
pick's slowdown against an on-the-spot exhaustive sweep of each op.  The metric is HBM GB/s of algorithmic traffic
(dot reads 8n bytes, scal reads 4n and writes 4n bytes; 16n per step) and
its fraction of the measured HBM peak.  Inputs (3 x 256 MiB) exceed the
129 MB L2, so no flush is needed between steps.

Other workloads (``--workload``): asum (n = 2^20; each call reads the next of
64 copies of x, twice the L2 in all, or with ``--submit eager`` the L2 is
flushed before every step), gemv_square (8192 x 8192), gemv_tall (65536 x 1024), mixed (bf16 and
fp8 asum / dot at 2^28), batch (20,000 ops), and more.  A default run (the
dot/scal workload on one GPU) also measures asum, both gemv shapes, mixed,
batch, both gemv-T shapes and BlackScholes after the headline step, each
with its own roofline, oracle check and CPU baseline, under ``config.sub``
(``--no-sub`` skips them).

Workloads whose step is a few plain calls (dot/scal, asum_large, gemv,
gemv-T, mixed, BlackScholes) submit their K timed steps as one CUDA graph
replay (``--submit graph``, the default: the calls run back to back with no
host launch between them, as a captured loop of calls runs); each call's
duration comes from a graph of K launches of that call alone, timed with
events on the replaying stream.  The same steps submitted one host call at a
time (events around each call) are reported in ``config.eager``.  The
batched dot/scal step (``--mode batched``) is one launch of the library's
own captured batch graph per step.

Under torchrun each rank runs its own replica on its own GPU (the ops of
one step do not exchange data); value is the bytes of all ranks divided by
the slowest rank's time.

``--impl reference`` times the CPU oracle instead (the FP64 pattern
interpreter on one host core): W warm-up and exactly K timed steps, each one
call of the oracle on the workload or its stated bounded slice.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "dot_scal": dict(n=1 << 26, desc="dot(x,y) + scal(1.5,x) fp32, n=2^26, N(0,1) seed 1"),
    "asum": dict(n=1 << 20, desc="asum(x) fp32, n=2^20, U(-1,1) seed 0, L2 flushed per step"),
    "asum_large": dict(n=1 << 26, desc="asum(x) fp32, n=2^26, N(0,1) seed 1"),
    "mixed": dict(n=1 << 28, desc="asum and dot on bf16 and on fp8-e4m3 (+ per-4096 scales), "
                                  "n=2^28, N(0,1) with 1% x1e3, seed 4"),
    "gemv_square": dict(M=8192, N=8192, desc="gemv fp32 8192x8192, alpha=1, beta=0.5, seed 2"),
    "gemv_tall": dict(M=65536, N=1024, desc="gemv fp32 65536x1024, alpha=1, beta=0.5, seed 2"),
    "gemv_t_square": dict(M=8192, N=8192, trans=True, desc="gemv-T (y = A^T x) fp32 8192x8192, alpha=1, "
                                               "beta=0.5, seed 5"),
    "gemv_t_tall": dict(M=65536, N=1024, trans=True, desc="gemv-T (y = A^T x) fp32 65536x1024, alpha=1, "
                                             "beta=0.5, seed 5"),
    "blackscholes": dict(n=1 << 26, desc="BlackScholes map (Fig. 6): 2^26 prices U(5,30), K=20, "
                                         "r=0.02, sigma=0.3, T=1, seed 6; call + put out"),
    "batch": dict(desc="batched launch: 20,000 ops (asum/dot/gemv, lengths 2^U(8,22), "
                       "gemv M,N 2^U(6,12)), about 60 GB, seed 3, one graph-launched "
                       "persistent kernel"),
}


E2E_CHUNKS = 8      # slices of the end-to-end pipeline (GB/s of dot + scal: 4 slices 336, 6: 304, 8: 347, 12: 299, 16: 310)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCE = {"asum": "reduce_f32.cuh", "dot": "reduce_f32.cuh", "nrm2": "reduce_f32.cuh",
                 "sum": "reduce_f32.cuh", "scal": "scal_gemv.cu",
                 "gemv": "scal_gemv.cu", "batch": "batch.cu", "mixed": "mixed.cu",
                 "gemv_tma": "gemv_tma.cu", "gemv_split": "gemv_split.cu", "gemv_t": "gemv_t.cu",
                 "blackscholes": "blackscholes.cu"}


def kernel_hash(tag: str) -> str:
    """Hash of the source of the kernel a tag names (its .cu file and the
    shared device header): ncu counters taken on other sources are stale."""
    if "bf16" in tag or "fp8" in tag:
        op = "mixed"
    elif tag.startswith("gemv_tma"):
        op = "gemv_tma"
    elif tag.startswith("gemv_split"):
        op = "gemv_split"
    elif tag.startswith("gemv_t_"):
        op = "gemv_t"
    else:
        op = tag.split("_", 1)[0]
    d = os.path.join(ROOT, "paper_1502_02389_gb300", "csrc")
    h = hashlib.sha256()
    for f in (KERNEL_SOURCE.get(op, ""), "lift_internal.cuh"):
        p = os.path.join(d, f)
        if f and os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:12]


def traffic_for(kernel_tag: str):
    """DRAM bytes per launch (read + write) from the committed ncu summary,
    when it was taken on the current source of that kernel
    ('variant-name source-hash bytes' lines of profiles/traffic.txt)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_hash(kernel_tag)
    for line in open(p):
        f = line.split()
        if len(f) == 3 and f[0] == kernel_tag and f[1] == want:
            return float(f[2])
    return None


def learned_gap(shapes, picked):
    """t(picked variant) / t(best variant) for each op of the step, all
    variants timed on the spot the way the autotuner times them (CUDA graph
    of back-to-back calls over cold slices, median of 5 replays)."""
    from paper_1502_02389_gb300 import lift, tune
    timer, pools = tune.Timer(), tune.Pools(seed=1)
    out = {}
    for (op, n, M, N) in shapes:
        buf = tune.Buffers(pools, op, n, M, N)
        times = {v: timer.per_call_ms([buf.call(v, r) for r in range(buf.R)], 5, 2)
                 for v in range(lift.lift_variant_count(op))}
        best = min(times, key=times.get)
        out[lift.OP_NAMES[op]] = {
            "picked": lift.lift_variant_describe(op, picked[op])["name"],
            "best": lift.lift_variant_describe(op, best)["name"],
            "ratio": round(times[picked[op]] / times[best], 4)}
    pools.cache.clear()
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (replicas: every rank runs its own copy of the
    step; the job is as fast as its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(bytes_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job GB/s: the bytes all ranks moved over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (max_ms / 1e3) / 1e9


BATCH_SCHEDULES = {"queue": 0, "per-item": 1}    # LIFT_BATCH_QUEUE, LIFT_BATCH_PER_ITEM


def batch_create(args, descs):
    """lift_batch_create, then the --batch-schedule choice (if any)."""
    from paper_1502_02389_gb300 import lift
    h = lift.lift_batch_create(descs)
    if getattr(args, "batch_schedule", None):
        lift.lift_batch_set_schedule(h, BATCH_SCHEDULES[args.batch_schedule])
    return h


def schedule_name(h):
    from paper_1502_02389_gb300 import lift
    k = lift.lift_batch_schedule(h)
    return {v: n for n, v in BATCH_SCHEDULES.items()}.get(k, str(k))


class Clocks:
    """nvidia-smi sampling (every 100 ms) around and during the timed
    region.  The sampler is started, and its first sample awaited, before
    the region opens, so that starting nvidia-smi does not overlap the
    timed work; the samples taken from just before the region to just after
    it are summarised (a region shorter than the sampling period is covered
    by its neighbouring samples)."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        import threading
        self.p = None
        self.lines = []
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.p = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t0 = time.monotonic()
        while not self.lines and time.monotonic() - t0 < 10.0 and self.p.poll() is None:
            time.sleep(0.01)
        self.t_start = time.monotonic()

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.monotonic(), line))

    def stop(self):
        if self.p is None:
            return None
        t_end = time.monotonic()
        while (not any(t > t_end for t, _ in self.lines) and time.monotonic() - t_end < 1.0
               and self.p.poll() is None):
            time.sleep(0.01)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            self.p.wait()
        self.reader.join(timeout=2)
        stamped = list(self.lines)
        before = [k for k, (t, _) in enumerate(stamped) if t <= self.t_start]
        lo = before[-1] if before else 0
        after = [k for k, (t, _) in enumerate(stamped) if t > t_end]
        hi = after[0] if after else len(stamped) - 1
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in stamped[lo:hi + 1]:
            f = [t.strip() for t in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_1502_02389_gb300 import build, lift, synth

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if local == 0:
        build.build()            # one builder per node; the other ranks wait for it
    if dist:
        dist.barrier()
    if local != 0:
        build.build()            # up to date by now: only checks timestamps
    lift.lift_init(local)
    dev = torch.device("cuda", local)
    wl = args.workload
    s = torch.cuda.current_stream()
    launches_per_step = 0
    kernels = []   # (tag, bytes per launch, start events, end events)
    # (kernels entry, launch of that call) for workloads whose step is a few
    # plain kernel calls: timed as CUDA graph replays (--submit graph)
    graph_calls = []
    flushed = False  # True: an L2 flush runs between the timed spans of each step
    collect = None   # after the timed steps: the GPU results the oracle leg checks
    pre_timed = None  # run once after the warm-up, before the timed region opens

    for name in args.variant or []:          # pin variants by name (profiling)
        for op in range(lift.NUM_OPS):
            ids = [v["id"] for v in lift.variants(op) if v["name"] == name]
            if ids:
                lift.lift_set_variant(op, ids[0])
                break
        else:
            raise SystemExit(f"unknown variant {name}")
    policy = "fixed"
    if wl != "batch" and not args.fixed_policy:
        from paper_1502_02389_gb300 import costmodel
        weights = args.mlp or costmodel.WEIGHTS
        if os.path.exists(weights):
            lift.lift_set_policy(lift.POLICY_MLP, weights)
            policy = "mlp"
    if wl == "dot_scal":
        n = WORKLOADS[wl]["n"]
        xh, yh, alpha = synth.dot_scal(n)
        x, y = torch.from_numpy(xh).to(dev), torch.from_numpy(yh).to(dev)
        z = torch.empty_like(x)
        r = torch.zeros(1, device=dev)
        vd = lift.lift_pick(lift.OP_DOT, n)
        vs = lift.lift_pick(lift.OP_SCAL, n)
        pd = lift.lift_variant_describe(lift.OP_DOT, vd)
        ps = lift.lift_variant_describe(lift.OP_SCAL, vs)
        bytes_step = 16 * n
        hb2 = batch_create(args, [
            {"op": lift.OP_DOT, "variant": vd, "n": n, "x": x, "y": y, "out": r},
            {"op": lift.OP_SCAL, "variant": vs, "n": n, "alpha": float(alpha), "x": x, "out": z}])

        def calls():
            lift.lift_dot_v(vd, x, y, n, r)
            lift.lift_scal_v(vs, n, float(alpha), x, z)

        if args.mode == "batched":
            launches_per_step = 1
            kb = ["batch:batch_dot_scal", bytes_step, [], []]
            kernels = [kb]

            def step(timed):
                if timed:
                    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev[0].record(s)
                lift.lift_batch_run(hb2)
                if timed:
                    ev[1].record(s)
                    kb[2].append(ev[0]); kb[3].append(ev[1])
        else:
            launches_per_step = pd["passes"] + 1
            kdot = ["dot:" + pd["name"], 8 * n, [], []]
            kscal = ["scal:" + ps["name"], 8 * n, [], []]
            kernels = [kdot, kscal]
            graph_calls = [(kdot, lambda: lift.lift_dot_v(vd, x, y, n, r)),
                           (kscal, lambda: lift.lift_scal_v(vs, n, float(alpha), x, z))]

            def step(timed):
                if timed:
                    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev[0].record(s)
                lift.lift_dot_v(vd, x, y, n, r)
                if timed:
                    ev2 = torch.cuda.Event(enable_timing=True)
                    ev[1].record(s)
                    kdot[2].append(ev[0]); kdot[3].append(ev[1])
                    ev2.record(s)
                lift.lift_scal_v(vs, n, float(alpha), x, z)
                if timed:
                    ev3 = torch.cuda.Event(enable_timing=True)
                    ev3.record(s)
                    kscal[2].append(ev2); kscal[3].append(ev3)

        # end to end: the step pipelined over E2E_CHUNKS slices of whole tiles
        # on three streams (host->device copies; the slice's dot partial and
        # scal; the device->host copy of its scal output), so the two copy
        # directions and the kernels overlap.  Each slice's dot goes to one
        # FP64 partial on the device (lift_dot_partial); after the last slice
        # the partials come back and lift_combine_partials adds them in slice
        # order and rounds once: the step returns the dot of the whole vectors.
        C = E2E_CHUNKS
        chunk = n // C
        parts64 = torch.zeros(C, dtype=torch.float64, device=dev)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(C)]
        ev_done = [torch.cuda.Event() for _ in range(C)]

        def e2e_step(xp, yp, zp, pp):
            s_in.wait_stream(s)
            for c in range(C):
                sl = slice(c * chunk, (c + 1) * chunk)
                with torch.cuda.stream(s_in):
                    x[sl].copy_(xp[sl], non_blocking=True)
                    y[sl].copy_(yp[sl], non_blocking=True)
                ev_in[c].record(s_in)
                s.wait_event(ev_in[c])
                lift.lift_dot_partial(x[sl], y[sl], chunk, parts64[c:c + 1], s)
                lift.lift_scal_v(vs, chunk, float(alpha), x[sl], z[sl], s)
                ev_done[c].record(s)
                s_out.wait_event(ev_done[c])
                with torch.cuda.stream(s_out):
                    zp[sl].copy_(z[sl], non_blocking=True)
            with torch.cuda.stream(s_out):
                pp.copy_(parts64, non_blocking=True)
            s.wait_stream(s_out)
            s_out.synchronize()
            return lift.lift_combine_partials(pp.tolist())[0]

        host = dict(xp=torch.from_numpy(xh).pin_memory(), yp=torch.from_numpy(yh).pin_memory(),
                    zp=torch.empty(n, dtype=torch.float32).pin_memory(),
                    pp=torch.empty(C, dtype=torch.float64).pin_memory())
        collect = lambda: {"dot": float(r.item()), "scal": z.cpu().numpy()}  # noqa: E731
        h2d, d2h = 8 * n, 4 * n + 8 * C
        config = {"workload": WORKLOADS[wl]["desc"], "n": n, "variants": [pd["name"], ps["name"]],
                  "submitted_as": ("one batched launch of the two calls (lift_batch_run)"
                                   if args.mode == "batched" else
                                   "two calls (lift_dot_v, lift_scal_v)"),
                  "l2": "no flush: inputs 3 x 256 MiB exceed the 129 MB L2"}
        if args.mode == "batched":
            config["batch_schedule"] = schedule_name(hb2)
    elif wl == "mixed":
        n = WORKLOADS[wl]["n"]
        xv, yv = synth.mixed_values(n)
        bx, by = synth.encode_bf16(xv), synth.encode_bf16(yv)
        (qx, sx), (qy, sy) = synth.encode_fp8_blocks(xv), synth.encode_fp8_blocks(yv)
        t = lambda a: torch.from_numpy(a).to(dev)  # noqa: E731
        bxd, byd, qxd, qyd, sxd, syd = t(bx), t(by), t(qx), t(qy), t(sx), t(sy)
        r = torch.zeros(4, device=dev)
        calls = []
        for name, op, dt, dargs, nb in (
                ("asum_bf16", lift.OP_ASUM_BF16, lift.BF16, (bxd, None), 2 * n),
                ("dot_bf16", lift.OP_DOT_BF16, lift.BF16, (bxd, None, byd, None), 4 * n),
                ("asum_fp8", lift.OP_ASUM_FP8, lift.FP8_E4M3, (qxd, sxd), n + 4 * sx.size),
                ("dot_fp8", lift.OP_DOT_FP8, lift.FP8_E4M3, (qxd, sxd, qyd, syd),
                 2 * n + 8 * sx.size)):
            v = lift.lift_pick(op, n)
            calls.append((op, dt, dargs, v, lift.lift_variant_describe(op, v)["name"], nb))
        kernels = [["mixed:" + name, nb, [], []] for (_, _, _, _, name, nb) in calls]
        bytes_step = sum(c[5] for c in calls)
        launches_per_step = 4

        def mixed_call(i):
            op, dt, da, v, name, nb = calls[i]
            if len(da) == 2:
                return lambda: lift.lift_asum_ex_v(v, dt, da[0], da[1], n, r[i:i + 1])
            return lambda: lift.lift_dot_ex_v(v, dt, da[0], da[1], da[2], da[3], n, r[i:i + 1])

        graph_calls = [(kernels[i], mixed_call(i)) for i in range(len(calls))]

        def step(timed):
            for i, (op, dt, da, v, name, nb) in enumerate(calls):
                if timed:
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(s)
                if len(da) == 2:
                    lift.lift_asum_ex_v(v, dt, da[0], da[1], n, r[i:i + 1])
                else:
                    lift.lift_dot_ex_v(v, dt, da[0], da[1], da[2], da[3], n, r[i:i + 1])
                if timed:
                    b.record(s)
                    kernels[i][2].append(a); kernels[i][3].append(b)

        e2e_step, host, h2d, d2h = None, {}, 0, 0
        collect = lambda: {"gpu": dict(zip(("asum_bf16", "dot_bf16", "asum_fp8", "dot_fp8"),  # noqa: E731
                                           r.cpu().numpy().tolist())),
                           "inputs": (xv, yv, bx, by, qx, sx, qy, sy)}
        config = {"workload": WORKLOADS[wl]["desc"], "n": n, "variants": [c[4] for c in calls],
                  "l2": "no flush: every input is at least 256 MiB"}
    elif wl == "asum_large":
        n = WORKLOADS[wl]["n"]
        xh, _, _ = synth.dot_scal(n)
        x = torch.from_numpy(xh).to(dev)
        r = torch.zeros(1, device=dev)
        va = lift.lift_pick(lift.OP_ASUM, n)
        pa = lift.lift_variant_describe(lift.OP_ASUM, va)
        launches_per_step = pa["passes"]
        bytes_step = 4 * n
        kas = ["asum:" + pa["name"], 4 * n, [], []]
        kernels = [kas]
        graph_calls = [(kas, lambda: lift.lift_asum_v(va, x, n, r))]

        def step(timed):
            if timed:
                ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev[0].record(s)
            lift.lift_asum_v(va, x, n, r)
            if timed:
                ev[1].record(s)
                kas[2].append(ev[0]); kas[3].append(ev[1])

        e2e_step, host, h2d, d2h = None, {}, 0, 0
        collect = lambda: {"asum": float(r.item())}  # noqa: E731
        config = {"workload": WORKLOADS[wl]["desc"], "n": n, "variants": [pa["name"]],
                  "l2": "no flush: x is 256 MiB, larger than the 129 MB L2"}
    elif wl == "asum":
        n = WORKLOADS[wl]["n"]
        xh = synth.asum_small(n)
        x = torch.from_numpy(xh).to(dev)
        r = torch.zeros(1, device=dev)
        flush = torch.ones(128 << 20, dtype=torch.float32, device=dev)
        va = lift.lift_pick(lift.OP_ASUM, n)
        pa = lift.lift_variant_describe(lift.OP_ASUM, va)
        launches_per_step = pa["passes"]
        bytes_step = 4 * n
        kas = ["asum:" + pa["name"], 4 * n, [], []]
        kernels = [kas]
        if args.submit == "graph":
            # cold data without a flush inside the timed region: every call
            # reads the next of ROT copies of x (ROT * 4 MiB = 256 MiB, twice
            # the L2), so a copy is read again only after 252 MiB of other
            # reads; the L2 is flushed once before the timed steps
            ROT = 64
            copies = x.repeat(ROT).view(ROT, n)
            nxt = [0]

            def rotating():
                lift.lift_asum_v(va, copies[nxt[0] % ROT], n, r)
                nxt[0] += 1

            graph_calls = [(kas, rotating)]

            def step(timed):
                if timed:
                    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev[0].record(s)
                rotating()
                if timed:
                    ev[1].record(s)
                    kas[2].append(ev[0]); kas[3].append(ev[1])
        else:
            def step(timed):
                flush.sum()     # read 512 MiB: evicts x from L2 and leaves no dirty lines
                if timed:
                    ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev[0].record(s)
                lift.lift_asum_v(va, x, n, r)
                if timed:
                    ev[1].record(s)
                    kas[2].append(ev[0]); kas[3].append(ev[1])

        def e2e_step(xp, rp):
            x.copy_(xp, non_blocking=True)
            lift.lift_asum_v(va, x, n, r)
            rp.copy_(r, non_blocking=True)

        host = dict(xp=torch.from_numpy(xh).pin_memory(), rp=torch.empty(1).pin_memory())
        collect = lambda: {"asum": float(r.item())}  # noqa: E731
        h2d, d2h = 4 * n, 4
        config = {"workload": WORKLOADS[wl]["desc"], "n": n, "variants": [pa["name"]]}
        if args.submit == "graph":
            config["l2"] = ("cold: every call reads the next of 64 copies of x (256 MiB in all, "
                            "twice the L2); the L2 flushed once before the timed steps")
            pre_timed = flush.sum
        else:
            config["l2"] = "flushed before every step (a 512 MiB read between the timed spans)"
            flushed = True
    elif wl == "blackscholes":
        n = WORKLOADS[wl]["n"]
        sh = synth.stock_prices(n)
        prm = (synth.BS_STRIKE, synth.BS_RATE, synth.BS_VOL, synth.BS_YEARS)
        sp = torch.from_numpy(sh).to(dev)
        call, put = torch.empty(n, device=dev), torch.empty(n, device=dev)
        vb = lift.lift_pick(lift.OP_BLACKSCHOLES, n)
        pb = lift.lift_variant_describe(lift.OP_BLACKSCHOLES, vb)
        launches_per_step = 1
        bytes_step = 12 * n
        kb = ["blackscholes:" + pb["name"], bytes_step, [], []]
        kernels = [kb]
        graph_calls = [(kb, lambda: lift.lift_blackscholes_v(vb, n, sp, *prm, call, put))]

        def step(timed):
            if timed:
                ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev[0].record(s)
            lift.lift_blackscholes_v(vb, n, sp, *prm, call, put)
            if timed:
                ev[1].record(s)
                kb[2].append(ev[0]); kb[3].append(ev[1])

        # end to end: pipelined over E2E_CHUNKS slices (prices in, the map,
        # calls and puts out on three streams)
        C = E2E_CHUNKS
        chunk = n // C
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(C)]
        ev_done = [torch.cuda.Event() for _ in range(C)]

        def e2e_step(sp_h, c_h, p_h):
            s_in.wait_stream(s)
            for c in range(C):
                sl = slice(c * chunk, (c + 1) * chunk)
                with torch.cuda.stream(s_in):
                    sp[sl].copy_(sp_h[sl], non_blocking=True)
                ev_in[c].record(s_in)
                s.wait_event(ev_in[c])
                lift.lift_blackscholes_v(vb, chunk, sp[sl], *prm, call[sl], put[sl], s)
                ev_done[c].record(s)
                s_out.wait_event(ev_done[c])
                with torch.cuda.stream(s_out):
                    c_h[sl].copy_(call[sl], non_blocking=True)
                    p_h[sl].copy_(put[sl], non_blocking=True)
            s.wait_stream(s_out)

        collect = lambda: {"call": call[:1 << 22].cpu().numpy(),  # noqa: E731
                           "put": put[:1 << 22].cpu().numpy()}
        host = dict(sp_h=torch.from_numpy(sh).pin_memory(), c_h=torch.empty(n).pin_memory(),
                    p_h=torch.empty(n).pin_memory())
        h2d, d2h = 4 * n, 8 * n
        config = {"workload": WORKLOADS[wl]["desc"], "n": n, "variants": [pb["name"]],
                  "options_per_s_note": "value / 12 bytes per option",
                  "l2": "no flush: 768 MiB moved per step, far beyond the 129 MB L2"}
    elif wl == "batch":
        from paper_1502_02389_gb300 import costmodel
        ops = synth.batch_ops()[:args.batch_ops]
        lay, total = synth.batch_layout(ops)
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        pool = torch.randn(total, device=dev, generator=g)
        base = pool.data_ptr()
        descs = []
        for d, e in zip(ops, lay):
            q = {"op": d["op"], "variant": -1, "n": d["n"], "M": d["M"], "N": d["N"],
                 "lda": d["N"], "alpha": 1.0, "beta": 0.5, "out": base + 4 * e["out"]}
            for k in ("x", "y", "A"):
                if k in e:
                    q[k] = base + 4 * e[k]
            descs.append(q)
        policies = {"fixed": (lift.POLICY_FIXED, None)}
        table = os.path.join(tempfile.gettempdir(), f"lift_bench_table_{os.getpid()}.txt")
        if not args.no_extras:          # the other policies, for comparison
            try:
                from paper_1502_02389_gb300 import tune
                recs = tune.load_csv(os.path.join(costmodel.DATA, "timings_gb300_train.csv"))
                os.makedirs(os.path.dirname(table), exist_ok=True)
                tune.write_table(recs, table)
                policies["table"] = (lift.POLICY_TABLE, table)
            except (OSError, AssertionError):
                pass
        weights = args.mlp or costmodel.WEIGHTS
        if os.path.exists(weights):
            policies["mlp"] = (lift.POLICY_MLP, weights)
            if args.no_extras:
                del policies["fixed"]
        handles = {}
        for name, (pol, path) in policies.items():
            lift.lift_set_policy(pol, path)
            handles[name] = batch_create(args, descs)
        lift.lift_set_policy(lift.POLICY_FIXED)
        main_policy = "mlp" if "mlp" in handles else "fixed"
        hb = handles[main_policy]
        info = lift.lift_batch_info(hb)
        bytes_step = info["bytes"]
        launches_per_step = 1
        kb = ["batch:batch_" + main_policy, bytes_step, [], []]
        kernels = [kb]

        def step(timed):
            if timed:
                ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev[0].record(s)
            lift.lift_batch_run(hb)
            if timed:
                ev[1].record(s)
                kb[2].append(ev[0]); kb[3].append(ev[1])

        # the other policies, timed the same way after the main measurement
        def policy_rates():
            out = {}
            for name, h in handles.items():
                for _ in range(2):
                    lift.lift_batch_run(h)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(s)
                for _ in range(5):
                    lift.lift_batch_run(h)
                b.record(s)
                torch.cuda.synchronize()
                out[name] = round(bytes_step * 5 / (a.elapsed_time(b) / 1e3) / 1e9, 1)
            return out

        # the oracle check: a fixed sample of ops; the sampled gemv outputs
        # (updated in place by every run) are put back to their initial
        # values and the batch run once more before they are read
        chk = np.sort(np.random.default_rng(7).choice(len(ops), min(200, len(ops)), replace=False))
        y0 = {int(i): pool[lay[i]["out"]:lay[i]["out"] + ops[i]["M"]].clone()
              for i in chk if ops[i]["op"] == synth.GEMV}

        def collect():
            for i, t in y0.items():
                pool[lay[i]["out"]:lay[i]["out"] + ops[i]["M"]].copy_(t)
            lift.lift_batch_run(hb)
            torch.cuda.synchronize()
            out = []
            for i in chk:
                d, e = ops[int(i)], lay[int(i)]
                get = lambda k, c: pool[e[k]:e[k] + c].cpu().numpy()  # noqa: E731
                if d["op"] == synth.GEMV:
                    out.append((d, {"A": get("A", d["M"] * d["N"]).reshape(d["M"], d["N"]),
                                    "x": get("x", d["N"]), "y0": y0[int(i)].cpu().numpy(),
                                    "got": get("out", d["M"])}))
                else:
                    out.append((d, {"x": get("x", d["n"]),
                                    "y": get("y", d["n"]) if d["op"] == synth.DOT else None,
                                    "got": float(pool[e["out"]].item())}))
            return {"ops": out, "of": len(ops)}

        e2e_step, host, h2d, d2h = None, {}, 0, 0
        config = {"workload": WORKLOADS[wl]["desc"], "ops": len(ops), "items": info["items"],
                  "grid": info["grid"], "policy": main_policy, "batch_schedule": schedule_name(hb),
                  "l2": "no flush: every run reads about 60 GB, far beyond the 129 MB L2"}
    else:
        M, N = WORKLOADS[wl]["M"], WORKLOADS[wl]["N"]
        trans = WORKLOADS[wl].get("trans", False)
        op, opname = (lift.OP_GEMV_T, "gemv_t") if trans else (lift.OP_GEMV, "gemv")
        call = lift.lift_gemv_t_v if trans else lift.lift_gemv_v
        Ah, xh, yh, a, b = synth.gemv_t(M, N) if trans else synth.gemv(M, N)
        nx, ny = (M, N) if trans else (N, M)
        A, xv, y0 = (torch.from_numpy(t).to(dev) for t in (Ah, xh, yh))
        yv = y0.clone()
        vg = lift.lift_pick(op, M * N, M, N)
        pg = lift.lift_variant_describe(op, vg)
        if trans:
            launches_per_step = pg["passes"]
        else:
            launches_per_step = 1 if lift.lift_gemv_segments(vg, M, N)[1] == 1 else 2
        bytes_step = 4 * M * N + 4 * nx + 8 * ny
        kg = [opname + ":" + pg["name"], bytes_step, [], []]
        kernels = [kg]
        graph_calls = [(kg, lambda: call(vg, M, N, float(a), A, N, xv, float(b), yv))]

        def step(timed):
            if timed:
                ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev[0].record(s)
            call(vg, M, N, float(a), A, N, xv, float(b), yv)
            if timed:
                ev[1].record(s)
                kg[2].append(ev[0]); kg[3].append(ev[1])

        def e2e_step(Ap, xp, yp, outp):
            A.copy_(Ap, non_blocking=True)
            xv.copy_(xp, non_blocking=True)
            yv.copy_(yp, non_blocking=True)
            call(vg, M, N, float(a), A, N, xv, float(b), yv)
            outp.copy_(yv, non_blocking=True)

        def collect():
            # one call on the initial y (the timed steps update y in place)
            y1 = y0.clone()
            call(vg, M, N, float(a), A, N, xv, float(b), y1)
            idx = np.sort(np.random.default_rng(5).choice(ny, 64, replace=False))
            return {"index": idx, "y": y1.cpu().numpy()[idx]}

        host = dict(Ap=torch.from_numpy(Ah).pin_memory(), xp=torch.from_numpy(xh).pin_memory(),
                    yp=torch.from_numpy(yh).pin_memory(), outp=torch.empty(ny).pin_memory())
        h2d, d2h = 4 * M * N + 4 * nx + 4 * ny, 4 * ny
        config = {"workload": WORKLOADS[wl]["desc"], "M": M, "N": N, "variants": [pg["name"]],
                  "l2": "no flush: A is 256 MiB, larger than the 129 MB L2"}

    use_graph = bool(graph_calls) and args.submit == "graph" and not flushed
    graphs = None
    if use_graph:
        # the K timed steps as one CUDA graph (calls back to back, as a loop
        # of calls submits them once captured), and per call a graph of K
        # launches of that call alone, which gives its average duration;
        # captured before the timed region, each replayed once untimed
        for _ in range(args.warmup):
            step(False)
        torch.cuda.synchronize()
        graphs = {"step": torch.cuda.CUDAGraph()}
        with torch.cuda.graph(graphs["step"]):
            for _ in range(args.steps):
                for _, fn in graph_calls:
                    fn()
        for i, (_, fn) in enumerate(graph_calls):
            graphs[i] = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graphs[i]):
                for _ in range(args.steps):
                    fn()
        for g in graphs.values():
            g.replay()
        torch.cuda.synchronize()
        config["submitted_as"] = (f"CUDA graph of the {args.steps} timed steps (calls back to "
                                  "back, no host launches); per-kernel time from a graph of "
                                  f"{args.steps} launches of that call alone")

    # ---- clock sampler up first (its start-up idles the GPU), then the
    # warm-up steps right before the K timed steps, which are bracketed by
    # barrier + synchronize
    clocks = Clocks(local) if rank == 0 else None
    for _ in range(args.warmup):
        if use_graph:
            graphs["step"].replay()
        else:
            step(False)
    if pre_timed is not None:
        pre_timed()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    if use_graph:
        graphs["step"].replay()
    else:
        for _ in range(args.steps):
            step(True)
    t1.record(s)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    bracket_ms = ms
    if flushed:
        # the L2 flush runs between timed iterations: the step time is the sum
        # of the per-step event spans, which bracket exactly the step's launches
        ms = sum(a.elapsed_time(b) for a, b in zip(kernels[0][2], kernels[0][3]))
        config["bracket_ms_including_flush"] = round(bracket_ms, 4)
    if use_graph:
        # per-call graphs: events on the stream that replays them
        for i, (ke, _) in enumerate(graph_calls):
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(s)
            graphs[i].replay()
            b_.record(s)
            torch.cuda.synchronize()
            per = a_.elapsed_time(b_) / args.steps
            ke[2].append(per)
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    value = job_rate(bytes_step, args.steps, world, ms)

    # ---- per-kernel durations (events on the launching stream)
    per_kernel = {}
    for tag, nbytes, starts, ends in kernels:
        if use_graph:
            d = list(starts)             # durations per launch from the per-call graph
        else:
            d = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        avg = sum(d) / len(d)
        per_kernel[tag] = {"ms": avg, "gbs": nbytes / (avg / 1e3) / 1e9, "bytes": nbytes}
    if use_graph:
        # the same steps submitted one call at a time, with events around each
        # call (context: the host launch path)
        for ke in kernels:
            ke[2].clear()
            ke[3].clear()
        for _ in range(3):
            step(False)
        # the step rate with events only around the K steps (a pair of events
        # around every call costs the stream a few microseconds itself), then
        # each call's duration from a second pass with events around each call
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_a.record(s)
        for _ in range(args.steps):
            step(False)
        e_b.record(s)
        torch.cuda.synchronize()
        eager_ms = e_a.elapsed_time(e_b)
        for _ in range(args.steps):
            step(True)
        torch.cuda.synchronize()
        config["eager"] = {
            "value": round(job_rate(bytes_step, args.steps, 1, eager_ms), 1),
            "kernels_gbs": {tag: round(nb / (sum(a.elapsed_time(b) for a, b in zip(st, en))
                                             / len(st) / 1e3) / 1e9, 1)
                            for tag, nb, st, en in kernels},
            "submitted_as": "one host call per op per step: value from events around the K steps, "
                            "kernels_gbs from a second pass with events around each call"}
        graphs = None
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    peak, src = peaks()
    tr = traffic_for(dom.split(":", 1)[1])
    roof = {"bound": "hbm", "achieved": round(per_kernel[dom]["gbs"], 1), "peak": peak,
            "unit": "GB/s", "frac": round(per_kernel[dom]["gbs"] / peak, 4),
            "traffic": tr, "kernel": dom, "peak_source": f"{src} hbm_gbs (copy bandwidth)",
            "algorithmic_bytes_per_launch": kernels[[k[0] for k in kernels].index(dom)][1]}

    # ---- end to end through the C-ABI with host buffers
    # (host clock around the steps, synchronised on both sides: the region
    # holds the copies, the kernels and any host-side finishing of a result)
    e2e = None
    if e2e_step is not None and not args.no_e2e:
        for _ in range(2):
            e2e_step(**host)
        torch.cuda.synchronize()
        ek = max(3, min(args.steps, 10))
        t_e = time.perf_counter()
        for _ in range(ek):
            e2e_result = e2e_step(**host)
        torch.cuda.synchronize()
        ems = (time.perf_counter() - t_e) * 1e3 / ek
        ems = max_over_ranks(ems, dist, dev)
        e2e = {"value": round(world * bytes_step / (ems / 1e3) / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ems, 4),
               "timer": "host clock, synchronised on both sides"}
        if e2e_result is not None:
            e2e["result"] = e2e_result
    if e2e is not None and wl in ("dot_scal", "blackscholes"):
        e2e["pipelined"] = f"{E2E_CHUNKS} slices; H2D, kernels and D2H on three streams"
    if e2e is not None and wl == "dot_scal":
        e2e["result_formed"] = ("dot of the whole vectors: FP64 slice partials "
                                "(lift_dot_partial) added by lift_combine_partials")
    if wl == "dot_scal" and args.no_extras:
        lift.lift_batch_destroy(hb2)
    elif wl == "dot_scal":
        config["policy"] = policy
        config["learned_vs_autotuned"] = learned_gap(
            [(lift.OP_DOT, n, 0, 0), (lift.OP_SCAL, n, 0, 0)], {lift.OP_DOT: vd, lift.OP_SCAL: vs})
        # context: the same step submitted the other way
        other = calls if args.mode == "batched" else (lambda: lift.lift_batch_run(hb2))
        for _ in range(3):
            other()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(s)
        for _ in range(50):
            other()
        b2.record(s)
        torch.cuda.synchronize()
        key = "same_step_as_two_calls_gbs" if args.mode == "batched" else \
            "same_step_as_one_batched_launch_gbs"
        config[key] = round(bytes_step * 50 / (a2.elapsed_time(b2) / 1e3) / 1e9, 1)
        lift.lift_batch_destroy(hb2)
    if wl == "batch" and not args.no_extras:
        config["policies_gbs"] = policy_rates()
    assert lift.lift_read_status() == 0
    results = collect() if (collect is not None and rank == 0) else None
    if wl == "batch":
        for h in handles.values():
            lift.lift_batch_destroy(h)
    if results is not None and e2e is not None and "result" in e2e:
        results["e2e_dot"] = e2e["result"]
    torch.cuda.synchronize()
    return dict(value=value, ms_step=ms_step, roofline=roof, per_kernel=per_kernel, clocks=clk,
                results=results,
                e2e=e2e, config=config, launches=launches_per_step * args.steps, peak=peak)


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
def oracle_work(workload: str):
    """One step of the oracle, as it stands, on the workload or a bounded
    slice of it: (work, algorithmic bytes of one call of work, description
    of the sample)."""
    import numpy as np

    from oracle import blas
    from paper_1502_02389_gb300 import synth

    if workload == "dot_scal":
        n = WORKLOADS[workload]["n"]
        x, y, alpha = synth.dot_scal(n)
        work = lambda: (blas.dot(x, y), blas.scal(float(alpha), x))  # noqa: E731
        bytes_one, what = 16 * n, f"full step (dot + scal, n=2^26)"
    elif workload == "asum_large":
        n = WORKLOADS[workload]["n"]
        x, _, _ = synth.dot_scal(n)
        work = lambda: blas.asum(x)  # noqa: E731
        bytes_one, what = 4 * n, "full step (asum, n=2^26)"
    elif workload == "mixed":
        from oracle import mixed
        n = 1 << 22
        xv, yv = synth.mixed_values(n)
        bx, by = synth.encode_bf16(xv), synth.encode_bf16(yv)
        (qx, sx), (qy, sy) = synth.encode_fp8_blocks(xv), synth.encode_fp8_blocks(yv)
        work = lambda: (mixed.asum("bf16", bx), mixed.dot("bf16", bx, None, by, None),  # noqa: E731
                        mixed.asum("fp8", qx, sx), mixed.dot("fp8", qx, sx, qy, sy))
        bytes_one = 2 * n + 4 * n + (n + 4 * sx.size) + (2 * n + 8 * sx.size)
        what = "the four mixed ops on the first 2^22 elements (same recipe, seed 4)"
    elif workload == "asum":
        n = WORKLOADS[workload]["n"]
        x = synth.asum_small(n)
        work = lambda: blas.asum(x)  # noqa: E731
        bytes_one, what = 4 * n, "full step (asum, n=2^20)"
    elif workload == "blackscholes":
        from oracle import finance
        n = 1 << 22
        sh = synth.stock_prices(WORKLOADS[workload]["n"])[:n]
        work = lambda: finance.black_scholes(sh, synth.BS_STRIKE, synth.BS_RATE,  # noqa: E731
                                             synth.BS_VOL, synth.BS_YEARS)
        bytes_one, what = 12 * n, "the first 2^22 prices (the paper's problem size)"
    elif workload == "batch":
        ops = synth.batch_ops()[:400]
        rng = np.random.default_rng(3)
        arrays = []
        for d in ops:
            if d["op"] == synth.GEMV:
                arrays.append((d, rng.standard_normal((d["M"], d["N"])), rng.standard_normal(d["N"]),
                               rng.standard_normal(d["M"])))
            else:
                arrays.append((d, rng.standard_normal(d["n"]),
                               rng.standard_normal(d["n"]) if d["op"] == synth.DOT else None, None))

        def work():
            for d, a1, a2, a3 in arrays:
                if d["op"] == synth.GEMV:
                    blas.gemv(a1, a2, a3, 1.0, 0.5)
                elif d["op"] == synth.DOT:
                    blas.dot(a1, a2)
                else:
                    blas.asum(a1)
        bytes_one = sum(4 * d["M"] * d["N"] + 4 * d["N"] + 8 * d["M"] if d["op"] == synth.GEMV
                        else (8 if d["op"] == synth.DOT else 4) * d["n"] for d in ops)
        what = "first 400 of the 20,000 batch ops (same op/size draws, host values)"
    elif WORKLOADS[workload].get("trans", False):
        M, N = WORKLOADS[workload]["M"], WORKLOADS[workload]["N"]
        A, xv, yv, a, b = synth.gemv_t(M, N)
        cols = max(1, N // 16)
        As, ys = np.ascontiguousarray(A[:, :cols]), yv[:cols]
        work = lambda: blas.gemv_t(As, xv, ys, float(a), float(b))  # noqa: E731
        bytes_one, what = 4 * M * cols + 4 * M + 8 * cols, f"first {cols} of {N} columns"
    else:
        M, N = WORKLOADS[workload]["M"], WORKLOADS[workload]["N"]
        A, xv, yv, a, b = synth.gemv(M, N)
        rows = max(1, M // 16)
        As, ys = A[:rows], yv[:rows]
        work = lambda: blas.gemv(As, xv, ys, float(a), float(b))  # noqa: E731
        bytes_one, what = 4 * rows * N + 4 * N + 8 * rows, f"first {rows} of {M} rows"
    return work, bytes_one, what


def oracle_sample(workload: str, budget_s: float):
    """Time the oracle, as it stands, on the workload (or a bounded slice of
    it) until about ``budget_s`` seconds of CPU work; returns GB/s of
    algorithmic bytes and a description of the sample."""
    work, bytes_one, what = oracle_work(workload)
    reps, t0 = 0, time.perf_counter()
    while True:
        work()
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el >= 30.0:
            break
    return bytes_one * reps / el / 1e9, f"{what}, {reps} repetition(s) in {el:.1f} s", el / reps


# ---- the oracle on every host core: contiguous fixed chunks of the step, one
# worker process per core (spawned, inputs in shared memory), the chunks'
# FP64 dots added in chunk order, so repeated runs give identical results
_MT = {}


def _mt_init(names, n):
    from multiprocessing import shared_memory

    import numpy as np
    shm = [shared_memory.SharedMemory(name=nm) for nm in names]
    _MT["shm"] = shm
    _MT["x"] = np.ndarray((n,), np.float32, buffer=shm[0].buf)
    _MT["y"] = np.ndarray((n,), np.float32, buffer=shm[1].buf)
    _MT["z"] = np.ndarray((n,), np.float64, buffer=shm[2].buf)


def _mt_chunk(task):
    from oracle import blas
    lo, hi, alpha = task
    x, y = _MT["x"][lo:hi], _MT["y"][lo:hi]
    _MT["z"][lo:hi] = blas.scal(alpha, x)
    return blas.dot(x, y)


def oracle_sample_threads(workload: str, budget_s: float):
    """The dot + scal step of the oracle on all host cores (see above);
    returns (GB/s, processes, sample description), or None for other
    workloads."""
    if workload != "dot_scal":
        return None
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np

    from paper_1502_02389_gb300 import synth
    n = WORKLOADS[workload]["n"]
    try:    # shared memory lives in /dev/shm: skip (None) where it is too small for 16n bytes
        st = os.statvfs("/dev/shm")
        if st.f_bavail * st.f_frsize < 16 * n + (256 << 20):
            return None
    except OSError:
        return None
    x, y, alpha = synth.dot_scal(n)
    procs = max(1, len(os.sched_getaffinity(0)))
    shm = [shared_memory.SharedMemory(create=True, size=n * sz) for sz in (4, 4, 8)]
    try:
        np.ndarray((n,), np.float32, buffer=shm[0].buf)[:] = x
        np.ndarray((n,), np.float32, buffer=shm[1].buf)[:] = y
        bounds = [n * k // procs for k in range(procs + 1)]
        tasks = [(bounds[k], bounds[k + 1], float(alpha)) for k in range(procs)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs, initializer=_mt_init, initargs=([m.name for m in shm], n)) as pool:
            pool.map(_mt_chunk, tasks)                      # warm-up: imports, page faults
            reps, t0 = 0, time.perf_counter()
            while True:
                parts = pool.map(_mt_chunk, tasks)
                sum(parts)                                  # the chunks' dots, in chunk order
                reps += 1
                el = time.perf_counter() - t0
                if el >= budget_s:
                    break
    finally:
        for m in shm:
            m.close()
            m.unlink()
    return (16 * n * reps / el / 1e9, procs,
            f"full step (dot + scal, n=2^26) in {procs} fixed contiguous chunks, one spawned "
            f"process per core, {reps} repetition(s) in {el:.1f} s")


def oracle_accuracy(workload: str, results):
    """The GPU results of the run against the oracle (the CPU leg): per result
    its absolute error and the parity bound (ratio <= 1: within the bound);
    scal is checked bit for bit.  None when the workload has no check here
    (the batch is checked op by op in the tests)."""
    import numpy as np

    from oracle import blas
    from paper_1502_02389_gb300 import synth

    if not results:
        return None

    def entry(got, ref, tol):
        err = abs(float(got) - float(ref))
        return {"abs_err": err, "tol": float(tol), "ratio": err / tol if tol > 0 else float(err > 0)}

    out = {}
    if workload == "dot_scal":
        n = WORKLOADS[workload]["n"]
        x, y, alpha = synth.dot_scal(n)
        ref, tol = blas.dot(x, y), blas.tolerance(n, blas.dot_terms(x, y))
        out["dot"] = entry(results["dot"], ref, tol)
        if results.get("e2e_dot") is not None:
            out["e2e_dot"] = entry(results["e2e_dot"], ref, tol)
        want = (np.float64(alpha) * x.astype(np.float64)).astype(np.float32)
        out["scal"] = {"bit_exact": bool(np.array_equal(results["scal"], want)), "elements": n}
    elif workload in ("asum", "asum_large"):
        n = WORKLOADS[workload]["n"]
        x = synth.asum_small(n) if workload == "asum" else synth.dot_scal(n)[0]
        out["asum"] = entry(results["asum"], blas.asum(x), blas.tolerance(n, blas.asum_terms(x)))
    elif workload == "mixed":
        from oracle import mixed
        n = WORKLOADS[workload]["n"]
        xv, yv, bx, by, qx, sx, qy, sy = results["inputs"]     # the draws and their encodings
        exact = {"asum": float(np.sum(np.abs(xv))), "dot": float(np.dot(xv, yv))}
        for dt, (ex, ey) in (("bf16", (mixed.stored_values("bf16", bx), mixed.stored_values("bf16", by))),
                             ("fp8", (mixed.stored_values("fp8", qx, sx),
                                      mixed.stored_values("fp8", qy, sy)))):
            for op in ("asum", "dot"):
                if op == "asum":
                    ref, terms = blas.asum(ex), float(np.sum(np.abs(ex)))
                else:
                    ref, terms = blas.dot(ex, ey), float(np.sum(np.abs(ex * ey)))
                e = entry(results["gpu"][f"{op}_{dt}"], ref, blas.tolerance(n, terms))
                e["quantisation_err"] = abs(ref - exact[op])      # stored values vs FP64 draws
                out[f"{op}_{dt}"] = e
            del ex, ey
    elif workload == "blackscholes":
        from oracle import finance
        m = 1 << 22
        s = synth.stock_prices(WORKLOADS[workload]["n"])[:m]
        prm = (synth.BS_STRIKE, synth.BS_RATE, synth.BS_VOL, synth.BS_YEARS)
        c, p = finance.black_scholes(s, *prm)
        tol = finance.tolerance(s, prm[0], prm[1], prm[3])
        for name, got, ref in (("call", results["call"], c), ("put", results["put"], p)):
            ratio = np.abs(got.astype(np.float64) - ref) / tol
            out[name] = {"max_abs_err": float(np.max(np.abs(got - ref))), "max_ratio": float(np.max(ratio)),
                         "options": m}
    elif workload == "batch":
        worst, count = 0.0, 0
        for d, a in results["ops"]:
            if d["op"] == synth.GEMV:
                A, x, y0 = (a[k].astype(np.float64) for k in ("A", "x", "y0"))
                ref = blas.gemv(A, x, y0, 1.0, 0.5)
                tol = blas.tolerance(d["N"], 1.0) * blas.gemv_row_terms(a["A"], a["x"], a["y0"], 1.0, 0.5)
                r = np.abs(a["got"].astype(np.float64) - ref) / tol
                worst = max(worst, float(np.max(r)) if r.size else 0.0)
            else:
                x = a["x"].astype(np.float64)
                if d["op"] == synth.ASUM:
                    ref, terms = blas.asum(x), blas.asum_terms(x)
                else:
                    y = a["y"].astype(np.float64)
                    ref, terms = blas.dot(x, y), blas.dot_terms(x, y)
                tol = blas.tolerance(d["n"], terms)
                worst = max(worst, abs(a["got"] - ref) / tol if tol > 0 else float(a["got"] != ref))
            count += 1
        out["ops"] = {"checked": count, "of": results["of"], "max_ratio": worst,
                      "sample": "fixed random sample (seed 7); every op in the GPU tests"}
    elif workload in ("gemv_square", "gemv_tall", "gemv_t_square", "gemv_t_tall"):
        M, N = WORKLOADS[workload]["M"], WORKLOADS[workload]["N"]
        idx = results["index"]
        if WORKLOADS[workload].get("trans", False):
            A, x, y, a, b = synth.gemv_t(M, N)
            As = A[:, idx].astype(np.float64)
            ref = blas.gemv_t(As, x.astype(np.float64), y[idx].astype(np.float64), float(a), float(b))
            terms = abs(float(a)) * (np.abs(As).T @ np.abs(x.astype(np.float64))) + \
                np.abs(float(b) * y[idx].astype(np.float64))
            n_red = M
        else:
            A, x, y, a, b = synth.gemv(M, N)
            ref = blas.gemv(A[idx].astype(np.float64), x.astype(np.float64), y[idx].astype(np.float64),
                            float(a), float(b))
            terms = blas.gemv_row_terms(A[idx], x, y[idx], float(a), float(b))
            n_red = N
        ratio = np.abs(results["y"].astype(np.float64) - ref) / (blas.tolerance(n_red, 1.0) * terms)
        out["y"] = {"max_ratio": float(np.max(ratio)), "sampled_outputs": int(idx.size)}
    else:
        return None
    return out


def run_reference(args):
    """The oracle as the reference arm: W untimed and exactly K timed steps,
    each step one call of the oracle on the workload (or its stated bounded
    slice), on one host core."""
    work, bytes_one, what = oracle_work(args.workload)
    for _ in range(args.warmup):
        work()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        work()
    el = time.perf_counter() - t0
    val = bytes_one * args.steps / el / 1e9
    sample = f"{what}; {args.steps} timed step(s) after {args.warmup} warm-up step(s), {el:.1f} s"
    out = {"metric": METRIC, "value": round(val, 4), "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(el / args.steps * 1e3, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOADS[args.workload]["desc"]},
           "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


METRIC = "HBM GB/s (frac of peak) for asum/dot/gemv; learned vs autotuned variant gap"

# the other configurations of the metric, measured in the same run after the
# headline step: asum at 2^20 (L2 flushed), both gemv shapes, the bf16 and fp8
# ops at 2^28, and the 20,000-op batched launch
SUB_WORKLOADS = ("asum", "gemv_square", "gemv_tall", "mixed", "batch", "gemv_t_square", "gemv_t_tall",
                 "blackscholes")


def run_subs(args, rank):
    """One record per SUB_WORKLOADS entry: K timed steps after W warm-up
    steps of that workload alone (its own CUDA events, roofline and clock
    samples), its results against the oracle, and the oracle timed on a
    short bounded sample of it."""
    import copy
    subs = {}
    for wl in SUB_WORKLOADS:
        sa = copy.copy(args)
        sa.workload, sa.no_e2e, sa.no_extras, sa.variant = wl, True, True, None
        t0 = time.perf_counter()
        r = run_ours(sa, rank, 1, None)
        val, sample, _ = oracle_sample(wl, budget_s=3.0)
        subs[wl] = {
            "workload": WORKLOADS[wl]["desc"], "value": round(r["value"], 2), "unit": "GB/s",
            "steps": sa.steps, "warmup": sa.warmup, "ms_per_step": round(r["ms_step"], 5),
            "frac_of_peak": round(r["value"] / r["peak"], 4), "roofline": r["roofline"],
            "kernels": {k: {"ms": round(v["ms"], 5), "gbs": round(v["gbs"], 1)}
                        for k, v in r["per_kernel"].items()},
            "gpu_launches": r["launches"], "clocks": r["clocks"], "config": r["config"],
            "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "accuracy_vs_oracle": oracle_accuracy(wl, r["results"])}
        subs[wl]["wall_s"] = round(time.perf_counter() - t0, 1)
    return subs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000,
                    help="timed steps (the default keeps the dot + scal region near 0.3 s, long enough for several clock samples)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dot_scal", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-schedule", default=None, choices=sorted(BATCH_SCHEDULES),
                    help="how batch work items meet the SMs (default: the library's)")
    ap.add_argument("--mlp", default=None, help="cost-model weights for the batch workload")
    ap.add_argument("--variant", action="append",
                    help="force a variant by name (repeatable), e.g. for a profiling capture")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--submit", default="graph", choices=["graph", "eager"],
                    help="single-call workloads: the timed steps as one CUDA graph replay "
                         "(default) or as host calls with events around each")
    ap.add_argument("--no-sub", action="store_true",
                    help="dot_scal: skip the records of the other configurations")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the on-the-spot variant sweep and the other submission mode")
    ap.add_argument("--mode", default="calls", choices=["batched", "calls"],
                    help="dot_scal: submit the step as two calls (default; with --submit graph "
                         "the timed steps run as one CUDA graph) or as one batched launch")
    ap.add_argument("--fixed-policy", action="store_true",
                    help="use the FIXED variant policy instead of the trained cost model")
    ap.add_argument("--batch-ops", type=int, default=20000,
                    help="ops of the batch workload (fewer only for profiling captures)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, dist)
    if rank == 0:
        cpu = None
        accuracy = None
        if world == 1 and not args.no_cpu_baseline:
            val, sample, _ = oracle_sample(args.workload, budget_s=10.0)
            cpu = {"value": round(val, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                   "sample": sample}
            mt = oracle_sample_threads(args.workload, budget_s=10.0)
            if mt is not None:
                cpu["all_cores"] = {"value": round(mt[0], 4), "unit": "GB/s", "cores": mt[1],
                                    "kind": "oracle", "sample": mt[2]}
            accuracy = oracle_accuracy(args.workload, res["results"])
        out = {"metric": METRIC, "value": round(res["value"], 2), "unit": "GB/s",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(res["ms_step"], 5), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": res["config"],
               "frac_of_peak": round(res["value"] / world / res["peak"], 4),
               "roofline": res["roofline"],
               "kernels": {k: {"ms": round(v["ms"], 5), "gbs": round(v["gbs"], 1)}
                           for k, v in res["per_kernel"].items()},
               "cpu_baseline": cpu, "e2e": res["e2e"], "clocks": res["clocks"],
               "gpu_launches": res["launches"], "accuracy_vs_oracle": accuracy}
        if world == 1 and args.workload == "dot_scal" and not args.no_sub and not args.variant:
            out["config"]["sub"] = run_subs(args, rank)
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
