"""The all-ops batch checker (tests/batch_oracle_pool.py) on the CPU: a
small batch laid out like the batched workload, its outputs computed as
fp32-rounded FP64 values, checked by spawned workers over double-buffered
shared memory in groups smaller than the batch; a planted wrong output in
each op kind is the only op flagged."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import batch_oracle_pool as bp
from paper_1502_02389_gb300 import synth


def test_checker_flags_exactly_the_planted_errors():
    ops = synth.batch_ops(count=90, lo=6, hi=12, mlo=3, mhi=7)
    lay, total = synth.batch_layout(ops)
    rng = np.random.default_rng(5)
    pool = rng.standard_normal(total).astype(np.float32)
    y0 = {}
    for i, (d, e) in enumerate(zip(ops, lay)):
        x = pool[e["x"]:e["x"] + (d["N"] if d["op"] == bp.GEMV else d["n"])].astype(np.float64)
        if d["op"] == bp.GEMV:
            A = pool[e["A"]:e["A"] + d["M"] * d["N"]].astype(np.float64).reshape(d["M"], d["N"])
            y = pool[e["out"]:e["out"] + d["M"]].copy()
            y0[i] = y
            pool[e["out"]:e["out"] + d["M"]] = (A @ x + 0.5 * y).astype(np.float32)
        elif d["op"] == bp.DOT:
            pool[e["out"]] = np.float32(x @ pool[e["y"]:e["y"] + d["n"]].astype(np.float64))
        else:
            pool[e["out"]] = np.float32(np.abs(x).sum())
    planted = {}
    for kind in (bp.ASUM, bp.DOT, bp.GEMV):
        i = next(j for j, d in enumerate(ops) if d["op"] == kind and j not in planted)
        planted[i] = kind
        pool[lay[i]["out"]] += np.float32(0.5)
    t = torch.from_numpy(pool)
    groups = list(bp._groups(ops, lay, total // 5))
    assert len(groups) >= 4                    # both buffers used, each more than once
    ratios, procs = bp.check_all(t, ops, lay, y0, chunk_bytes=4 * (total // 5))
    assert procs >= 1 and sorted(ratios) == list(range(len(ops)))
    bad = sorted(i for i, r in ratios.items() if r > 1.0)
    assert bad == sorted(planted)
