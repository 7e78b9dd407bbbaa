"""nrm2, sum and axpy: user functions through the same kernel templates,
against the oracle's programs (tolerance at n = 2^26, bit for bit against
each variant's low-level expression on ragged sizes, axpy bit-exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas
from oracle import lowlevel as ll
from oracle.patterns import evaluate
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


def _run(L, op, vid, xd, n):
    r = torch.full((1,), -7.0, device="cuda")
    r64 = torch.full((1,), -7.0, device="cuda", dtype=torch.float64)
    (L.lift_nrm2_v if op == "nrm2" else L.lift_sum_v)(vid, xd, n, r, r64)
    torch.cuda.synchronize()
    return np.float32(r.item()), float(r64.item())


def test_full_size_all_variants(L):
    x, y, _ = synth.dot_scal()
    n = x.size
    x64 = x.astype(np.float64)
    ref_n, ref_s = blas.nrm2(x64), blas.sum_(x64)
    tol_n = blas.nrm2_tolerance(n, float((x64 * x64).sum()))
    tol_s = blas.tolerance(n, blas.asum_terms(x))
    xd = torch.from_numpy(x).cuda()
    for op, OP, ref, tol in (("nrm2", L.OP_NRM2, ref_n, tol_n), ("sum", L.OP_SUM, ref_s, tol_s)):
        for vid in range(L.lift_variant_count(OP)):
            got, got64 = _run(L, op, vid, xd, n)
            assert abs(float(got) - ref) <= tol, (op, vid, got, ref, tol)
    r = torch.zeros(1, device="cuda")
    L.lift_nrm2(xd, n, r)
    assert abs(float(r.item()) - ref_n) <= tol_n


@pytest.mark.parametrize("n", [1, 33, 4097, 70001])
def test_bit_exact_to_expression(L, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    for op, OP in (("nrm2", L.OP_NRM2), ("sum", L.OP_SUM)):
        for vid in range(L.lift_variant_count(OP)):
            v = L.lift_variant_describe(OP, vid)
            g = L.lift_variant_grid(OP, vid, n)
            e, Lp = ll.reduce_variant(op, n, v["tile"], v["vw"], v["threads"], g, bool(v["stride"]),
                                      v["cluster"], v["final_threads"])
            xp = np.zeros(Lp, np.float32)
            xp[:n] = x
            exp = evaluate(e, xp, mode="f32")[0]
            got, _ = _run(L, op, vid, xd, n)
            assert got == exp, (v["name"], n, got, exp)


def test_axpy_bit_exact_all_variants(L):
    x, y, _ = synth.dot_scal()
    exp = blas.axpy(-0.75, x, y, mode="f32")                # fl(fl(a x) + y), oracle fp32 mode
    xd = torch.from_numpy(x).cuda()
    for vid in range(L.lift_variant_count(L.OP_AXPY)):
        yd = torch.from_numpy(y).cuda()
        L.lift_axpy_v(vid, x.size, -0.75, xd, yd)
        assert np.array_equal(yd.cpu().numpy().view(np.uint32), exp.view(np.uint32))
    # ragged, unaligned and in place
    for n in (1, 1023, 70001):
        xs = np.random.default_rng(n).standard_normal(n).astype(np.float32)
        for vid in range(L.lift_variant_count(L.OP_AXPY)):
            buf = torch.zeros(n + 8, device="cuda")
            buf[1:n + 1] = torch.from_numpy(xs).cuda()
            L.lift_axpy_v(vid, n, 2.0, buf.data_ptr() + 4, buf.data_ptr() + 4)   # y == x
            got = buf[1:n + 1].cpu().numpy()
            assert np.array_equal(got, blas.axpy(2.0, xs, xs, mode="f32"))
            assert buf[0].item() == 0 and torch.all(buf[n + 1:] == 0)


def test_empty(L):
    r = torch.full((1,), 3.0, device="cuda")
    x = torch.zeros(4, device="cuda")
    L.lift_nrm2(x, 0, r)
    assert r.item() == 0.0
    L.lift_sum(x, 0, r)
    assert r.item() == 0.0
