"""The device-side timeout path, exercised without a fault: a wait that
nothing satisfies gives up after its poll limit, the status word reports
LIFT_ERR_TIMEOUT, reading it clears it, and the context stays usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    return lift


def test_wait_gives_up_and_reports(L):
    assert L.lift_read_status(1) == 0
    t = time.perf_counter()
    L.lift_wait_probe(256)
    torch.cuda.synchronize()
    assert time.perf_counter() - t < 5.0
    assert L.lift_read_status(1) == L.ERR_TIMEOUT       # reported ...
    assert L.lift_read_status(1) == 0                   # ... and cleared by the read
    # the context is still usable: a staged (bulk-copy) variant computes correctly
    x = np.random.default_rng(0).standard_normal(1 << 20).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    r = torch.empty(1, device="cuda")
    vid = [v["id"] for v in L.variants(L.OP_ASUM) if v["stages"] > 0][0]
    L.lift_asum_v(vid, xd, x.size, r)
    assert abs(r.item() - blas.asum(x)) <= blas.tolerance(x.size, blas.asum_terms(x))
    assert L.lift_read_status(1) == 0


def test_probe_arguments(L):
    with pytest.raises(L.LiftError):
        L.lift_wait_probe(0)
    with pytest.raises(L.LiftError):
        L.lift_wait_probe((1 << 22) + 1)


def _expected_bits(L, opname, op, vid, x, y):
    """The variant's low-level expression evaluated in fp32 mode."""
    from oracle import lowlevel as ll
    from oracle.patterns import evaluate
    v = L.lift_variant_describe(op, vid)
    n = x.size
    e, Lp = ll.reduce_variant(opname, n, v["tile"], v["vw"], v["threads"],
                              L.lift_variant_grid(op, vid, n), bool(v["stride"]), v["cluster"],
                              v["final_threads"])
    xp = np.zeros(Lp, np.float32)
    xp[:n] = x
    if opname != "dot":
        return np.float32(evaluate(e, xp, mode="f32")[0])
    yp = np.zeros(Lp, np.float32)
    yp[:n] = y
    return np.float32(evaluate(e, (xp, yp), mode="f32")[0])


def _run(L, opname, vid, xd, yd, n, r):
    if opname == "asum":
        L.lift_asum_v(vid, xd, n, r)
    elif opname == "dot":
        L.lift_dot_v(vid, xd, yd, n, r)
    elif opname == "nrm2":
        L.lift_nrm2_v(vid, xd, n, r)
    else:
        L.lift_sum_v(vid, xd, n, r)


def test_staged_reduction_timeout_keeps_the_one_pass_tickets(L):
    """A real staged reduction driven down its timeout path: with the wait
    limit at 0 every CTA's first wait on a bulk copy gives up, so the call
    records LIFT_ERR_TIMEOUT, drains its copies and returns NaN -- and,
    because every CTA still takes its "last CTA" ticket, the ticket is back
    at 0.  The very next one-pass asum / dot / nrm2 / sum calls (before the
    status word is read, so nothing resets the tickets for them) equal their
    low-level expressions bit for bit."""
    assert L.lift_read_status(1) == 0
    n = 70001
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    r = torch.empty(1, device="cuda")
    ops = (("asum", L.OP_ASUM), ("dot", L.OP_DOT), ("nrm2", L.OP_NRM2), ("sum", L.OP_SUM))
    staged = [(nm, op, v["id"]) for nm, op in ops for v in L.variants(op)
              if v["stages"] > 0 and v["passes"] == 1]
    assert staged
    L.lift_set_wait_polls(0)
    try:
        for nm, op, vid in staged:
            r.fill_(1.0)
            _run(L, nm, vid, xd, yd, n, r)
            torch.cuda.synchronize()
            assert np.isnan(r.item()), L.lift_variant_describe(op, vid)["name"]
    finally:
        L.lift_set_wait_polls(1 << 22)
    for nm, op in ops:
        for v in L.variants(op):
            if v["passes"] != 1:
                continue
            r.fill_(-7.0)
            _run(L, nm, v["id"], xd, yd, n, r)
            torch.cuda.synchronize()
            got = np.float32(r.item())
            assert got == _expected_bits(L, nm, op, v["id"], x, y), v["name"]
    assert L.lift_read_status(1) == L.ERR_TIMEOUT
    assert L.lift_read_status(1) == 0


def test_wait_polls_arguments(L):
    with pytest.raises(L.LiftError):
        L.lift_set_wait_polls((1 << 22) + 1)
    L.lift_set_wait_polls(1 << 22)


def test_staged_gemv_t_timeout(L):
    """The staged gemv-T forms driven down their timeout path: with the wait
    limit at 0 the consumer warps give up on their first stage and the
    producer on its first reuse of a stage; both wait (with the full limit)
    for the copies in flight, the partials are NaN, so every y_j is NaN and
    the status word reads LIFT_ERR_TIMEOUT.  With the limit restored the same
    calls match the two-pass expression bit for bit."""
    from oracle import lowlevel as ll
    from oracle.patterns import evaluate
    assert L.lift_read_status(1) == 0
    M, N = 3000, 1100                     # several stages per block, a ragged column block
    rng = np.random.default_rng(12)
    A = rng.standard_normal((M, N)).astype(np.float32)
    x = rng.standard_normal(M).astype(np.float32)
    Ad, xd = torch.from_numpy(A).cuda(), torch.from_numpy(x).cuda()
    staged = [v for v in L.variants(L.OP_GEMV_T) if v["stages"] > 0]
    assert staged
    L.lift_set_wait_polls(0)
    try:
        for v in staged:
            yd = torch.zeros(N, device="cuda")
            L.lift_gemv_t_v(v["id"], M, N, 1.0, Ad, N, xd, 0.0, yd)
            torch.cuda.synchronize()
            assert torch.isnan(yd).all().item(), v["name"]
    finally:
        L.lift_set_wait_polls(1 << 22)
    assert L.lift_read_status(1) == L.ERR_TIMEOUT
    for v in staged:
        B, RB = L.lift_gemv_t_blocks(v["id"], M, N)
        z = evaluate(ll.gemv_t_z_variant(M, N, 1.0, B, RB, 2), A, mode="f32", env={"x": x})
        yd = torch.zeros(N, device="cuda")
        L.lift_gemv_t_v(v["id"], M, N, 1.0, Ad, N, xd, 0.0, yd)
        assert np.array_equal(yd.cpu().numpy(), z.astype(np.float32)), v["name"]
    assert L.lift_read_status(1) == 0
