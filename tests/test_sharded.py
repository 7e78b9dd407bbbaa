"""Sharded reductions over ranks (world size 2, gloo, CPU): each rank reduces
its shard to one FP64 partial, the ranks all-gather the 8-byte partials and
combine them with the library's host-side lift_combine_partials; every rank
gets the same result, within the parity bound of the whole-vector oracle.
The shard partials here come from the oracle (no GPU in these tests); the
GPU test test_gpu_sharded.py makes them with lift_asum_partial."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    from oracle import blas
    from paper_1502_02389_gb300 import lift, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = (1 << 20) + 13
        x, y, _ = synth.dot_scal(n)
        cut = [0, 400000, n][rank:rank + 2]           # uneven shards
        xs, ys = x[cut[0]:cut[1]], y[cut[0]:cut[1]]
        mine = torch.tensor([blas.asum(xs), blas.dot(xs, ys)], dtype=torch.float64)
        parts = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, mine)                   # the one exchange: 16 bytes per rank
        a = lift.lift_combine_partials([float(p[0]) for p in parts])
        d = lift.lift_combine_partials([float(p[1]) for p in parts])
        q.put((rank, a, d, blas.asum(x), blas.tolerance(n, blas.asum_terms(x)),
               blas.dot(x, y), blas.tolerance(n, blas.dot_terms(x, y))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_their_partials():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]      # same result on every rank
    for _, (a, a64), (d, d64), ea, ta, ed, td in res:
        assert abs(a - ea) <= ta and abs(d - ed) <= td
        assert a == np.float32(a64) and d == np.float32(d64)


def test_combine_is_the_ordered_fp64_sum():
    from paper_1502_02389_gb300 import lift
    r, r64 = lift.lift_combine_partials([2.0 ** 60, 1.0, -(2.0 ** 60), 0.25])
    assert r64 == (((2.0 ** 60 + 1.0) - 2.0 ** 60) + 0.25) and r == np.float32(r64)
    assert lift.lift_combine_partials([]) == (0.0, 0.0)
