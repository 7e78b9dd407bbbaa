"""The full batched workload (20,000 asum / dot / gemv ops, about 60 GB in
one device pool, the policy's variants, one graph-launched persistent
kernel): after one run, every op's operands are read back and checked
against the FP64 oracle within the parity bound -- all 20,000, on every
host core (tests/batch_oracle_pool.py)."""
import time

import pytest

torch = pytest.importorskip("torch")

from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu


def test_every_op_of_the_batched_workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import batch_oracle_pool as bp
    from paper_1502_02389_gb300 import build, costmodel, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    ops = synth.batch_ops()
    lay, total = synth.batch_layout(ops)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    pool = torch.randn(total, device="cuda", generator=g)
    base = pool.data_ptr()
    descs = []
    for d, e in zip(ops, lay):
        q = {"op": d["op"], "variant": -1, "n": d["n"], "M": d["M"], "N": d["N"], "lda": d["N"],
             "alpha": 1.0, "beta": 0.5, "out": base + 4 * e["out"]}
        for k in ("x", "y", "A"):
            if k in e:
                q[k] = base + 4 * e[k]
        descs.append(q)
    y0 = {i: pool[e["out"]:e["out"] + d["M"]].cpu().numpy()
          for i, (d, e) in enumerate(zip(ops, lay)) if d["op"] == synth.GEMV}
    lift.lift_set_policy(lift.POLICY_MLP, costmodel.WEIGHTS)
    try:
        h = lift.lift_batch_create(descs)
    finally:
        lift.lift_set_policy(lift.POLICY_FIXED)
    try:
        lift.lift_batch_run(h)
        torch.cuda.synchronize()
        assert lift.lift_read_status() == 0
        t = time.perf_counter()
        ratios, procs = bp.check_all(pool, ops, lay, y0)
        print(f"20,000 ops checked on {procs} processes in {time.perf_counter() - t:.1f} s; "
              f"worst ratio {max(ratios.values()):.3g}")
    finally:
        lift.lift_batch_destroy(h)
    assert len(ratios) == len(ops) == 20000
    bad = {i: r for i, r in ratios.items() if not r <= 1.0}
    assert not bad, (len(bad), sorted(bad.items())[:10])
