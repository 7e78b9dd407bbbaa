"""Calls chained on one stream with no host synchronisation in between.

Most kernels of the library are launched as programmatic dependents of the
kernel before them on the stream: a call's CTAs may be scheduled while the
previous call is still running, and each waits (griddepcontrol.wait) before
its first global memory access.  This test chains calls of every family that
is launched that way -- scal and axpy in place, asum / dot / nrm2 / sum in
one and two passes, the compensated and mixed-precision reductions, gemv,
gemv-T and BlackScholes -- so that each call reads what the call before it
wrote (read after write) or overwrites what the call before it read (write
after read, including the shared partials and "last CTA" tickets of
consecutive reductions), cycling through every variant of each op.  The
results must be the bits of the same chain run with a synchronisation after
every call, and so must a CUDA graph of the chain replayed from the same
start."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu

N_VEC = (1 << 22) + 37        # ragged vectors
M, N = 2048, 1024             # gemv / gemv-T (whole 16-byte rows: every variant runs as itself)
N_MIX = (1 << 20) + 4099      # bf16 / fp8 inputs
N_BS = (1 << 20) + 3          # options
SLOTS = 9                     # results per round


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    yield lift
    torch.cuda.synchronize()
    assert lift.lift_read_status() == 0


def _start():
    """Initial host state of every buffer the chain reads or writes."""
    w = synth.asum_small(N_VEC, seed=21)
    v = synth.asum_small(N_VEC, seed=22)
    A, _, g, _, _ = synth.gemv(M, N, seed=23)
    xm, ym = synth.mixed_values(N_MIX, seed=24)
    q1, s1 = synth.encode_fp8_blocks(xm)
    q2, s2 = synth.encode_fp8_blocks(ym)
    return dict(w=w, v=v, A=np.ascontiguousarray(A, np.float32), g=g.astype(np.float32),
                xb=synth.encode_bf16(xm), q1=q1, s1=s1, q2=q2, s2=s2,
                p=synth.stock_prices(N_BS, seed=25))


class Chain:
    def __init__(self, L, host, rounds):
        self.L = L
        self.host = host
        self.d = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in host.items()}
        self.res = torch.zeros(rounds * SLOTS, device="cuda")
        self.call = torch.zeros(N_BS, device="cuda")
        self.put = torch.zeros(N_BS, device="cuda")
        self.cs = torch.zeros(N_BS, device="cuda")
        self.rounds = rounds
        cnt = {op: L.lift_variant_count(op) for op in range(L.NUM_OPS)}
        self.vid = lambda op, r: r % cnt[op]

    def reset(self):
        for k, a in self.host.items():
            self.d[k].copy_(torch.from_numpy(np.ascontiguousarray(a)))
        self.res.zero_()
        self.call.zero_()
        self.put.zero_()
        self.cs.zero_()
        torch.cuda.synchronize()

    def issue(self, s, sync):
        L, d, v = self.L, self.d, self.vid
        w, vv, A, g = d["w"], d["v"], d["A"], d["g"]

        def step(f):
            f()
            if sync:
                s.synchronize()

        for r in range(self.rounds):
            o = lambda k: self.res[r * SLOTS + k: r * SLOTS + k + 1]
            step(lambda: L.lift_scal_v(v(L.OP_SCAL, r), N_VEC, 0.75, w, w, s))
            step(lambda: L.lift_asum_v(v(L.OP_ASUM, r), w, N_VEC, o(0), None, s))
            step(lambda: L.lift_axpy_v(v(L.OP_AXPY, r), N_VEC, 0.5, vv, w, s))
            step(lambda: L.lift_dot_v(v(L.OP_DOT, r), w, vv, N_VEC, o(1), None, s))
            step(lambda: L.lift_asum_v(v(L.OP_ASUM, r + 7), w, N_VEC, o(2), None, s))
            step(lambda: L.lift_gemv_v(v(L.OP_GEMV, r), M, N, 1.0 / 64, A, N, w, 0.5, g, s))
            step(lambda: L.lift_gemv_t_v(v(L.OP_GEMV_T, r), M, N, 1.0 / 128, A, N, g, 0.25, w, s))
            step(lambda: L.lift_nrm2_v(v(L.OP_NRM2, r), w, N_VEC, o(3), None, s))
            step(lambda: L.lift_sum_v(v(L.OP_SUM, r), w, N_VEC, o(4), None, s))
            step(lambda: L.lift_asum_comp_v(v(L.OP_ASUM_COMP, r), w, N_VEC, o(5), None, s))
            step(lambda: L.lift_dot_comp_v(v(L.OP_DOT_COMP, r), w, vv, N_VEC, o(6), None, s))
            step(lambda: L.lift_asum_ex_v(v(L.OP_ASUM_BF16, r), L.BF16, d["xb"], None, N_MIX, o(7),
                                          None, s))
            step(lambda: L.lift_dot_ex_v(v(L.OP_DOT_FP8, r), L.FP8_E4M3, d["q1"], d["s1"], d["q2"],
                                         d["s2"], N_MIX, o(8), None, s))
            step(lambda: L.lift_blackscholes_v(v(L.OP_BLACKSCHOLES, r), N_BS, d["p"], synth.BS_STRIKE,
                                               synth.BS_RATE, synth.BS_VOL, synth.BS_YEARS,
                                               self.call, self.put, s))
            step(lambda: L.lift_scal_v(v(L.OP_SCAL, r + 3), N_BS, 1.25, self.call, self.cs, s))

    def state(self):
        torch.cuda.synchronize()
        out = {k: self.d[k] for k in ("w", "g")}
        out.update(res=self.res, call=self.call, put=self.put, cs=self.cs)
        return {k: t.cpu().numpy().view(np.uint32).copy() for k, t in out.items()}


def test_chain_without_syncs_and_as_a_graph_matches_synchronised_calls(L):
    host = _start()
    rounds = max(L.lift_variant_count(op) for op in (L.OP_ASUM, L.OP_DOT, L.OP_SCAL, L.OP_GEMV,
                                                     L.OP_GEMV_T))
    ch = Chain(L, host, rounds)
    s = torch.cuda.Stream()

    ch.reset()
    ch.issue(s, sync=True)
    want = ch.state()
    assert np.isfinite(want["res"].view(np.float32)).all()
    assert np.isfinite(want["w"].view(np.float32)).all()

    ch.reset()
    ch.issue(s, sync=False)
    got = ch.state()
    for k in want:
        assert np.array_equal(got[k], want[k]), k

    ch.reset()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ch.issue(s, sync=False)
    ch.reset()                      # capture ran nothing; start again from the same state
    graph.replay()
    got = ch.state()
    for k in want:
        assert np.array_equal(got[k], want[k]), k
