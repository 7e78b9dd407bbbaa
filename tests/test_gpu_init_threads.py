"""lift_init called from several host threads at once sets the device up
once: the workspace is allocated a single time (device memory in use grows
by one workspace, not one per thread), the calls that follow give the
oracle's result, and a lift_finalize followed by another burst of
concurrent lift_init calls does the same again.  It runs in a fresh process
so that finalising the library disturbs no other test."""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = textwrap.dedent(
    """
    import threading
    import numpy as np
    import torch
    from oracle import blas
    from paper_1502_02389_gb300 import build, lift, synth

    build.build()
    torch.cuda.set_device(0)
    torch.cuda.synchronize()
    x = synth.asum_small((1 << 20) + 333, seed=11)
    xd = torch.from_numpy(x).cuda()
    r = torch.empty(1, device="cuda")
    tol = blas.tolerance(x.size, blas.asum_terms(x))
    want = blas.asum(x.astype(np.float64))

    def burst(k):
        errs = []
        go = threading.Barrier(k)

        def one():
            try:
                go.wait()
                lift.lift_init(0)
            except Exception as e:          # reported by the parent
                errs.append(repr(e))

        ts = [threading.Thread(target=one) for _ in range(k)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errs, errs

    used = []
    for rep in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        burst(8)
        torch.cuda.synchronize()
        used.append(free0 - torch.cuda.mem_get_info()[0])
        lift.lift_asum(xd, x.size, r)
        torch.cuda.synchronize()
        assert abs(float(r) - want) <= tol, (float(r), want)
        assert lift.lift_read_status() == 0
        lift.lift_finalize()
    print("USED", used)
    """
)


def test_concurrent_lift_init_sets_up_once():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = subprocess.run([sys.executable, "-c", _CHILD], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    line = [l for l in p.stdout.splitlines() if l.startswith("USED")][-1]
    used = [int(v) for v in line[4:].strip(" []").split(",")]
    # one workspace: 8 slots of 16 MiB fp32 + 1 MiB FP64 partials and the
    # ticket counters (about 138 MiB); a second set-up would double it
    one = 8 * ((1 << 22) * 4 + (1 << 17) * 8 + (64 + 65536) * 4)
    for u in used:
        assert u < 1.5 * one, (u, one)
