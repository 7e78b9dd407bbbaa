"""Reductions on several streams at once: each stream has its own workspace
slot (partials and "last CTA" tickets), so one-pass and two-pass asum /
dot, the compensated and fp8 reductions and gemv-T, issued interleaved on
four streams, give exactly the results of the same calls made one after
another on one stream."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu


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


def _calls(L, k, data, out):
    """The calls of stream k: (result slot, thunk taking a stream)."""
    x, y, A, xa, q, sc, n, M, N = data[k]
    calls = []
    for v in L.variants(L.OP_ASUM)[::5]:
        calls.append(lambda s, r, v=v: L.lift_asum_v(v["id"], x, n, r, None, s))
    for v in L.variants(L.OP_DOT)[::5]:
        calls.append(lambda s, r, v=v: L.lift_dot_v(v["id"], x, y, n, r, None, s))
    for v in L.variants(L.OP_DOT_COMP):
        calls.append(lambda s, r, v=v: L.lift_dot_comp_v(v["id"], x, y, n, r, None, s))
    for v in L.variants(L.OP_ASUM_FP8)[:4]:
        calls.append(lambda s, r, v=v: L.lift_asum_ex_v(v["id"], L.FP8_E4M3, q, sc, n, r, None, s))
    return calls


def test_interleaved_streams_match_serial(L):
    rng = np.random.default_rng(4)
    streams = [torch.cuda.Stream() for _ in range(4)]
    data = []
    for k in range(4):
        n = (1 << 22) + 977 * k
        xh = rng.standard_normal(n).astype(np.float32)
        yh = rng.standard_normal(n).astype(np.float32)
        qh, sh = synth.encode_fp8_blocks(xh.astype(np.float64))
        M, N = 3000 + 17 * k, 2048
        Ah = rng.standard_normal((M, N)).astype(np.float32)
        xah = rng.standard_normal(M).astype(np.float32)
        t = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
        data.append((t(xh), t(yh), t(Ah), t(xah), t(qh), t(sh), n, M, N))
    ncalls = len(_calls(L, 0, data, None))
    gt_variants = [v["id"] for v in L.variants(L.OP_GEMV_T)]
    res = torch.full((4, ncalls), float("nan"), device="cuda")
    ys = [torch.zeros((len(gt_variants), data[k][8]), device="cuda") for k in range(4)]
    torch.cuda.synchronize()
    # interleaved: call i of every stream before call i + 1 of any
    per = [_calls(L, k, data, None) for k in range(4)]
    for i in range(ncalls):
        for k, s in enumerate(streams):
            per[k][i](s, res[k, i:i + 1])
    for j, vid in enumerate(gt_variants):
        for k, s in enumerate(streams):
            _, _, A, xa, _, _, _, M, N = data[k]
            L.lift_gemv_t_v(vid, M, N, 1.0, A, N, xa, 0.0, ys[k][j], s)
    torch.cuda.synchronize()
    # serial, on one stream
    ref = torch.full((4, ncalls), float("nan"), device="cuda")
    yr = [torch.zeros_like(ys[k]) for k in range(4)]
    s0 = torch.cuda.current_stream()
    for k in range(4):
        for i, c in enumerate(per[k]):
            c(s0, ref[k, i:i + 1])
        _, _, A, xa, _, _, _, M, N = data[k]
        for j, vid in enumerate(gt_variants):
            L.lift_gemv_t_v(vid, M, N, 1.0, A, N, xa, 0.0, yr[k][j], s0)
    torch.cuda.synchronize()
    assert torch.equal(res, ref)
    for k in range(4):
        assert torch.equal(ys[k], yr[k])
