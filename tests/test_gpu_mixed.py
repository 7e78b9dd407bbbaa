"""GPU parity of the mixed-precision asum / dot (bf16, fp8-e4m3 with block
scales) against the FP64 oracle on the stored values.

The mixed workload: n = 2^28, N(0,1) with 1 % of entries scaled by 1e3
(seed 4).  Each result must satisfy |gpu - oracle(stored)| <=
4 u log2(n) sum|terms(stored)|; the quantisation error (oracle on stored
values vs oracle on the FP64 draws) is reported beside it.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas, mixed
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(L, op, vid, dt, x, xs, y=None, ys=None, n=None, offset=0):
    n = x.size if n is None else n
    esz = x.dtype.itemsize
    xd = torch.zeros(x.nbytes + 64 * esz, dtype=torch.uint8, device="cuda")
    xd[offset * esz: offset * esz + x.nbytes] = dev(x.view(np.uint8))
    r = torch.zeros(1, device="cuda")
    r64 = torch.zeros(1, device="cuda", dtype=torch.float64)
    xsd = dev(xs) if xs is not None else None
    if y is None:
        L.lift_asum_ex_v(vid, dt, xd.data_ptr() + offset * esz, xsd, n, r, r64)
    else:
        yd = torch.zeros(y.nbytes + 64 * esz, dtype=torch.uint8, device="cuda")
        yd[offset * esz: offset * esz + y.nbytes] = dev(y.view(np.uint8))
        ysd = dev(ys) if ys is not None else None
        L.lift_dot_ex_v(vid, dt, xd.data_ptr() + offset * esz, xsd, yd.data_ptr() + offset * esz,
                        ysd, n, r, r64)
    torch.cuda.synchronize()
    return float(r.item()), float(r64.item())


@pytest.fixture(scope="module")
def workload():
    n = 1 << 28
    xv, yv = synth.mixed_values(n)
    out = {"n": n, "x64": xv, "y64": yv}
    out["bf16"] = (synth.encode_bf16(xv), synth.encode_bf16(yv))
    out["fp8"] = (synth.encode_fp8_blocks(xv), synth.encode_fp8_blocks(yv))
    return out


def _cases(L, w):
    bx, by = w["bf16"]
    (qx, sx), (qy, sy) = w["fp8"]
    return [
        ("asum_bf16", L.OP_ASUM_BF16, L.BF16, (bx, None, None, None), lambda: mixed.asum("bf16", bx),
         lambda: blas.asum(w["x64"]), lambda v: np.abs(v).sum()),
        ("dot_bf16", L.OP_DOT_BF16, L.BF16, (bx, None, by, None), lambda: mixed.dot("bf16", bx, None, by, None),
         lambda: blas.dot(w["x64"], w["y64"]), None),
        ("asum_fp8", L.OP_ASUM_FP8, L.FP8_E4M3, (qx, sx, None, None), lambda: mixed.asum("fp8", qx, sx),
         lambda: blas.asum(w["x64"]), None),
        ("dot_fp8", L.OP_DOT_FP8, L.FP8_E4M3, (qx, sx, qy, sy), lambda: mixed.dot("fp8", qx, sx, qy, sy),
         lambda: blas.dot(w["x64"], w["y64"]), None),
    ]


def test_mixed_full_size_all_variants(L, workload):
    n = workload["n"]
    bx, by = workload["bf16"]
    (qx, sx), (qy, sy) = workload["fp8"]
    report = []
    for name, op, dt, (x, xs, y, ys), ref_stored, ref_orig, _ in _cases(L, workload):
        ref = ref_stored()
        vx = mixed.stored_values("bf16" if dt == L.BF16 else "fp8", x, xs)
        if y is None:
            terms = float(np.abs(vx).sum())
        else:
            vy = mixed.stored_values("bf16" if dt == L.BF16 else "fp8", y, ys)
            terms = float(np.abs(vx * vy).sum())
            del vy
        del vx
        tol = blas.tolerance(n, terms)
        quant = abs(ref - ref_orig())
        for vid in range(L.lift_variant_count(op)):
            got, got64 = run(L, op, vid, dt, x, xs, y, ys)
            acc_err = abs(got - ref)
            assert acc_err <= tol, (name, vid, got, ref, tol)
            assert abs(got64 - ref) <= tol
            report.append((name, L.lift_variant_describe(op, vid)["name"], acc_err / terms,
                           quant / terms))
    for r in report:
        print("%-10s %-24s accumulation err/sum|t| = %.3e  quantisation err/sum|t| = %.3e" % r)


@pytest.mark.parametrize("n", [0, 1, 17, 4095, 4096, 4097, 100003])
def test_mixed_ragged_sizes(L, n):
    xv, yv = synth.mixed_values(max(n, 1), seed=100 + n)
    xv, yv = xv[:n], yv[:n]
    bx, by = synth.encode_bf16(xv), synth.encode_bf16(yv)
    (qx, sx), (qy, sy) = synth.encode_fp8_blocks(xv), synth.encode_fp8_blocks(yv)
    if n == 0:
        sx = sy = np.ones(1, np.float32)
        bx = by = np.zeros(1, np.uint16)
        qx = qy = np.zeros(1, np.uint8)
    cases = [(L.OP_ASUM_BF16, L.BF16, bx, None, None, None, lambda: mixed.asum("bf16", bx[:n])),
             (L.OP_DOT_BF16, L.BF16, bx, None, by, None,
              lambda: mixed.dot("bf16", bx[:n], None, by[:n], None)),
             (L.OP_ASUM_FP8, L.FP8_E4M3, qx, sx, None, None, lambda: mixed.asum("fp8", qx[:n], sx)),
             (L.OP_DOT_FP8, L.FP8_E4M3, qx, sx, qy, sy,
              lambda: mixed.dot("fp8", qx[:n], sx, qy[:n], sy))]
    for op, dt, x, xs, y, ys, ref_fn in cases:
        ref = ref_fn() if n else 0.0
        kind = "bf16" if dt == L.BF16 else "fp8"
        vx = mixed.stored_values(kind, x[:n], xs)
        terms = float(np.abs(vx * mixed.stored_values(kind, y[:n], ys)).sum()) if y is not None \
            else float(np.abs(vx).sum())
        for vid in range(L.lift_variant_count(op)):
            for off in (0, 1):      # off = 1 element: unaligned -> guarded form
                got, _ = run(L, op, vid, dt, x, xs, y, ys, n=n, offset=off)
                assert abs(got - ref) <= blas.tolerance(max(n, 1), terms), (op, vid, off, got, ref)


def test_mixed_nan_and_inf(L):
    n = 10000
    bx = synth.encode_bf16(np.ones(n))
    bx[777] = 0x7F80                        # +Inf in bf16
    got, _ = run(L, L.OP_ASUM_BF16, 0, L.BF16, bx, None)
    assert got == math.inf
    bx[778] = 0xFF80                        # -Inf: dot with ones gives +Inf + -Inf = NaN
    got, _ = run(L, L.OP_DOT_BF16, 0, L.BF16, bx, None, synth.encode_bf16(np.ones(n)), None)
    assert math.isnan(got)
    q, s = synth.encode_fp8_blocks(np.ones(n))
    q[5000] = 0x7F                          # E4M3 NaN
    got, _ = run(L, L.OP_ASUM_FP8, 0, L.FP8_E4M3, q, s)
    assert math.isnan(got)
