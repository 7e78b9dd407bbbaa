"""Read guards (the other half of the memory checks without a sanitizer):
every input is placed inside a buffer whose surrounding words -- and, for
matrices, the columns between N and the leading dimension -- hold NaN.  A
kernel that reads past its input and folds what it read into a result turns
that result into NaN (0 * NaN is NaN too), so every variant of every
reading op must return finite values within the parity bound, with ragged
sizes, misaligned starts and padded leading dimensions.  Nothing here can
fault: the NaN words are inside the same allocation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas, mixed
from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu
PAD = 64


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


def nan_padded(a, off=0, fill=np.nan):
    """Device copy of the 1-D array a, starting `off` elements after PAD
    elements of `fill`, followed by PAD more; returns (buffer, address)."""
    a = np.ascontiguousarray(a)
    h = np.full(a.size + 2 * PAD + off, fill, dtype=a.dtype)
    h[PAD + off:PAD + off + a.size] = a
    d = torch.from_numpy(h.view(np.uint8) if a.dtype.itemsize != 4 else h).cuda()
    return d, d.data_ptr() + (PAD + off) * a.dtype.itemsize


def padded_matrix(A, lda, off=0):
    """A (M x N, fp32) stored row-major with leading dimension lda; the
    columns N..lda and the words around the matrix hold NaN."""
    M, N = A.shape
    h = np.full((M, lda), np.nan, np.float32)
    h[:, :N] = A
    return nan_padded(h.reshape(-1), off)


def vals(n, seed):
    return np.random.default_rng(seed).uniform(1.0, 2.0, n).astype(np.float32)


@pytest.mark.parametrize("n,off", [(1, 0), (4099, 1), (262147, 3), (1 << 20, 0)])
def test_reductions_read_only_their_inputs(L, n, off):
    x, y = vals(n, 1), vals(n, 2)
    bx, px = nan_padded(x, off)
    by, py = nan_padded(y, off)
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    cases = [
        (L.OP_ASUM, lambda v, r: L.lift_asum_v(v, px, n, r), blas.asum(x64), blas.asum_terms(x)),
        (L.OP_DOT, lambda v, r: L.lift_dot_v(v, px, py, n, r), blas.dot(x64, y64),
         blas.dot_terms(x, y)),
        (L.OP_SUM, lambda v, r: L.lift_sum_v(v, px, n, r), float(np.sum(x64)), blas.asum_terms(x)),
        (L.OP_NRM2, lambda v, r: L.lift_nrm2_v(v, px, n, r), float(np.sqrt(np.sum(x64 * x64))),
         None),
        (L.OP_ASUM_COMP, lambda v, r: L.lift_asum_comp_v(v, px, n, r), blas.asum(x64),
         blas.asum_terms(x)),
        (L.OP_DOT_COMP, lambda v, r: L.lift_dot_comp_v(v, px, py, n, r), blas.dot(x64, y64),
         blas.dot_terms(x, y)),
    ]
    for op, call, ref, terms in cases:
        tol = blas.tolerance(n, terms) if terms is not None else \
            (4 * max(1, int(np.ceil(np.log2(n)))) + 2) * 2.0 ** -24 * ref
        for vid in range(L.lift_variant_count(op)):
            r = torch.full((1,), -1.0, device="cuda")
            call(vid, r)
            got = float(r.item())
            name = L.lift_variant_describe(op, vid)["name"]
            assert np.isfinite(got), (name, n, off)
            assert abs(got - ref) <= tol, (name, n, off, got, ref)


@pytest.mark.parametrize("M,N,lda,off", [(1, 1, 1, 0), (37, 1030, 1032, 1), (3000, 64, 72, 0),
                                         (5, 70000, 70004, 2), (37, 1280, 1536, 0),
                                         (11, 512, 515, 0), (700, 257, 260, 3)])
def test_matrix_ops_read_only_their_inputs(L, M, N, lda, off):
    A = vals(M * N, 3).reshape(M, N)
    bA, pA = padded_matrix(A, lda, off)
    A64 = A.astype(np.float64)
    for op, rows, cols, call in ((L.OP_GEMV, M, N, L.lift_gemv_v), (L.OP_GEMV_T, N, M, L.lift_gemv_t_v)):
        x = vals(cols, 4)
        y0 = vals(rows, 5)
        bx, px = nan_padded(x, off)
        x64, y64 = x.astype(np.float64), y0.astype(np.float64)
        if op == L.OP_GEMV:
            ref = blas.gemv(A64, x64, y64, 1.0, 0.5)
            terms = blas.gemv_row_terms(A, x, y0, 1.0, 0.5)
            n_red = N
        else:
            ref = blas.gemv_t(A64, x64, y64, 1.0, 0.5)
            terms = np.abs(A64).T @ np.abs(x64) + np.abs(0.5 * y64)
            n_red = M
        tol = blas.tolerance(n_red, 1.0) * terms
        for vid in range(L.lift_variant_count(op)):
            y = torch.from_numpy(y0.copy()).cuda()
            call(vid, M, N, 1.0, pA, lda, px, 0.5, y)
            got = y.cpu().numpy()
            name = L.lift_variant_describe(op, vid)["name"]
            assert np.all(np.isfinite(got)), (name, M, N, lda, off)
            assert np.all(np.abs(got - ref) <= tol), (name, M, N, lda, off)


@pytest.mark.parametrize("n,off", [(4097, 0), (100003, 0), (100003, 1)])
def test_mixed_read_only_their_inputs(L, n, off):
    xv, yv = synth.mixed_values(n, seed=21)
    bx16, by16 = synth.encode_bf16(xv), synth.encode_bf16(yv)
    (qx, sx), (qy, sy) = synth.encode_fp8_blocks(xv), synth.encode_fp8_blocks(yv)
    nan16, nan8 = np.uint16(0x7FC0), np.uint8(0x7F)       # NaN in bf16 and in e4m3
    cases = [
        ("bf16", L.BF16, bx16, by16, None, None, nan16),
        ("fp8", L.FP8_E4M3, qx, qy, sx, sy, nan8),
    ]
    for kind, dt, x, y, xs, ys, nanv in cases:
        bxd, px = nan_padded(x, off, fill=nanv)
        byd, py = nan_padded(y, off, fill=nanv)
        keep = [bxd, byd]                  # the device buffers stay alive while the kernels run
        if xs is not None:
            bxs, pxs = nan_padded(xs)
            bys, pys = nan_padded(ys)
            keep += [bxs, bys]
        else:
            pxs = pys = None
        vx = mixed.stored_values(kind, x, xs)
        vy = mixed.stored_values(kind, y, ys)
        for op, call, ref, terms in (
                (L.OP_ASUM_BF16 if kind == "bf16" else L.OP_ASUM_FP8,
                 lambda v, r: L.lift_asum_ex_v(v, dt, px, pxs, n, r),
                 mixed.asum(kind, x, xs), float(np.abs(vx).sum())),
                (L.OP_DOT_BF16 if kind == "bf16" else L.OP_DOT_FP8,
                 lambda v, r: L.lift_dot_ex_v(v, dt, px, pxs, py, pys, n, r),
                 mixed.dot(kind, x, xs, y, ys), float(np.abs(vx * vy).sum()))):
            for vid in range(L.lift_variant_count(op)):
                r = torch.full((1,), -1.0, device="cuda")
                call(vid, r)
                got = float(r.item())
                name = L.lift_variant_describe(op, vid)["name"]
                assert np.isfinite(got), (name, n, off)
                assert abs(got - ref) <= blas.tolerance(n, terms), (name, n, off, got, ref)


@pytest.mark.parametrize("schedule", [0, 1])      # LIFT_BATCH_QUEUE, LIFT_BATCH_PER_ITEM
def test_batch_reads_only_its_inputs(L, schedule):
    """A batch of asum / dot / gemv ops of ragged sizes and misaligned starts,
    each operand between NaN words (gemv: and NaN in the lda padding)."""
    rng = np.random.default_rng(9)
    descs, checks, keep = [], [], []
    for i in range(60):
        kind = i % 3
        off = i % 4
        if kind < 2:
            n = int(rng.choice([1, 31, 4097, 70001, 300003]))
            x, y = vals(n, 100 + i), vals(n, 200 + i)
            bx, px = nan_padded(x, off)
            by, py = nan_padded(y, off)
            out = torch.full((1,), -1.0, device="cuda")
            keep += [bx, by, out]
            d = {"op": L.OP_ASUM if kind == 0 else L.OP_DOT, "variant": -1, "n": n, "x": px,
                 "out": out}
            if kind == 0:
                ref, terms = blas.asum(x.astype(np.float64)), blas.asum_terms(x)
            else:
                d["y"] = py
                ref, terms = blas.dot(x.astype(np.float64), y.astype(np.float64)), blas.dot_terms(x, y)
            descs.append(d)
            checks.append((out, ref, blas.tolerance(n, terms)))
        else:
            M, N = int(rng.integers(1, 200)), int(rng.choice([1, 33, 128, 1000, 4100]))
            lda = N + int(rng.choice([0, 3, 8]))
            A = vals(M * N, 300 + i).reshape(M, N)
            x, y0 = vals(N, 400 + i), vals(M, 500 + i)
            bA, pA = padded_matrix(A, lda, off)
            bx, px = nan_padded(x, off)
            y = torch.from_numpy(y0.copy()).cuda()
            keep += [bA, bx, y]
            descs.append({"op": L.OP_GEMV, "variant": -1, "M": M, "N": N, "lda": lda,
                          "alpha": 1.0, "beta": 0.5, "A": pA, "x": px, "out": y})
            ref = blas.gemv(A.astype(np.float64), x.astype(np.float64), y0.astype(np.float64),
                            1.0, 0.5)
            checks.append((y, ref, blas.tolerance(N, 1.0) * blas.gemv_row_terms(A, x, y0, 1.0, 0.5)))
    h = L.lift_batch_create(descs)
    try:
        L.lift_batch_set_schedule(h, schedule)
        L.lift_batch_run(h)
        torch.cuda.synchronize()
        for i, (out, ref, tol) in enumerate(checks):
            got = out.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got)), i
            assert np.all(np.abs(got - ref) <= tol), i
    finally:
        L.lift_batch_destroy(h)
