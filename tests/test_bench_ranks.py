"""bench.py's multi-rank arithmetic on CPU ranks (gloo, world size 2): each
rank runs its own replica, the job time is the slowest rank's, and the
whole-job rate counts the bytes of every rank."""
import os
import socket

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
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.0, 30.0][rank]          # rank 1 is slower
        dist.barrier()
        got = bench.max_over_ranks(ms, dist, "cpu")
        q.put((rank, got, bench.job_rate(1e9, 10, world, got)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, got, rate in res:
        assert got == 30.0
        assert abs(rate - 2 * 1e9 * 10 / 0.030 / 1e9) < 1e-9


def test_single_rank_rate():
    import bench
    assert bench.max_over_ranks(5.0, None, "cpu") == 5.0
    assert bench.job_rate(16 * 2 ** 26, 100, 1, 181.0) == pytest.approx(16 * 2 ** 26 * 100 / 0.181 / 1e9)
