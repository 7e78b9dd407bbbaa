"""GPU parity of the fp32 asum / dot / scal / gemv kernels against the CPU
oracle, through the C-ABI.

Three kinds of check:
  * tolerance: |gpu - oracle_fp64| <= 4 u log2(n) sum|terms| for every
    variant at the workload sizes (asum n = 2^20, dot/scal n = 2^26, gemv
    8192 x 8192 and 65536 x 1024 on sampled rows);
  * bit-exact: each variant equals its own low-level expression evaluated
    by the oracle in fp32-rounded mode (small ragged sizes), which pins the
    split, reorder-stride, vector width, tree and combine structure;
  * scal is bit-exact against the correctly rounded product everywhere.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas
from oracle import lowlevel as ll
from oracle.patterns import C, Map, Zip, add, evaluate, mult_by
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


def reduce_gpu(L, op, vid, x, y=None, offset=0):
    n = x.size
    xd = torch.zeros(n + offset + 8, device="cuda")
    xd[offset:offset + n] = dev(x)
    r = torch.full((1,), -7.0, device="cuda")
    r64 = torch.full((1,), -7.0, device="cuda", dtype=torch.float64)
    if op == "asum":
        L.lift_asum_v(vid, xd.data_ptr() + 4 * offset, n, r, r64)
    else:
        yd = torch.zeros(n + offset + 8, device="cuda")
        yd[offset:offset + n] = dev(y)
        L.lift_dot_v(vid, xd.data_ptr() + 4 * offset, yd.data_ptr() + 4 * offset, n, r, r64)
    torch.cuda.synchronize()
    return np.float32(r.item()), float(r64.item())


def expected_bits(L, opname, vid, x, y=None):
    """Evaluate the variant's low-level expression in fp32 mode."""
    op = L.OP_ASUM if opname == "asum" else L.OP_DOT
    v = L.lift_variant_describe(op, vid)
    n = x.size
    g = L.lift_variant_grid(op, vid, n)
    e, Lp = ll.reduce_variant(opname, n, v["tile"], v["vw"], v["threads"], g, bool(v["stride"]),
                              v["cluster"], v["final_threads"])
    e64, _ = ll.reduce_variant(opname, n, v["tile"], v["vw"], v["threads"], g, bool(v["stride"]),
                               v["cluster"], v["final_threads"], cast32=False)
    xp = np.zeros(Lp, np.float32)
    xp[:n] = x
    if opname == "asum":
        return evaluate(e, xp, mode="f32")[0], float(evaluate(e64, xp, mode="f32")[0])
    yp = np.zeros(Lp, np.float32)
    yp[:n] = y
    return evaluate(e, (xp, yp), mode="f32")[0], float(evaluate(e64, (xp, yp), mode="f32")[0])


# ---------------------------------------------------------------------------
# asum (n = 2^20, U(-1,1), seed 0) and dot (n = 2^26, N(0,1), seed 1)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def asum_case():
    x = synth.asum_small()
    return x, blas.asum(x.astype(np.float64)), blas.asum_terms(x)


@pytest.fixture(scope="module")
def dot_case():
    x, y, alpha = synth.dot_scal()
    ref = blas.dot(x.astype(np.float64), y.astype(np.float64))
    return x, y, float(alpha), ref, blas.dot_terms(x, y)


def test_asum_all_variants_full_size(L, asum_case):
    x, ref, terms = asum_case
    tol = blas.tolerance(x.size, terms)
    for vid in range(L.lift_variant_count(L.OP_ASUM)):
        got, got64 = reduce_gpu(L, "asum", vid, x)
        assert abs(float(got) - ref) <= tol, (L.lift_variant_describe(L.OP_ASUM, vid)["name"], got, ref)
        assert abs(got64 - ref) <= tol


def test_dot_all_variants_full_size(L, dot_case):
    x, y, _, ref, terms = dot_case
    n = x.size
    tol = blas.tolerance(n, terms)
    xd, yd = dev(x), dev(y)
    r = torch.zeros(1, device="cuda")
    for vid in range(L.lift_variant_count(L.OP_DOT)):
        r.fill_(-7.0)
        L.lift_dot_v(vid, xd, yd, n, r)
        got = float(r.item())
        assert abs(got - ref) <= tol, (L.lift_variant_describe(L.OP_DOT, vid)["name"], got, ref, tol)


def test_asum_default_entry_point(L, asum_case):
    x, ref, terms = asum_case
    xd = dev(x)
    r = torch.zeros(1, device="cuda")
    L.lift_asum(xd, x.size, r)
    assert abs(float(r.item()) - ref) <= blas.tolerance(x.size, terms)


@pytest.mark.parametrize("n", [1, 2, 33, 4097, 70001])
def test_reduce_variants_bit_exact_to_their_expression(L, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    for opname, op in (("asum", L.OP_ASUM), ("dot", L.OP_DOT)):
        for vid in range(L.lift_variant_count(op)):
            got, got64 = reduce_gpu(L, opname, vid, x, y)
            exp, exp64 = expected_bits(L, opname, vid, x, y)
            name = L.lift_variant_describe(op, vid)["name"]
            assert got == exp, (name, n, got, exp)
            assert got64 == exp64, (name, n, got64, exp64)


def test_misaligned_pointers_use_the_guarded_form(L):
    n = 50001
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    ref_a = blas.asum(x.astype(np.float64))
    ref_d = blas.dot(x.astype(np.float64), y.astype(np.float64))
    for opname, op in (("asum", L.OP_ASUM), ("dot", L.OP_DOT)):
        for vid in range(L.lift_variant_count(op)):
            got, _ = reduce_gpu(L, opname, vid, x, y, offset=1)   # 4-byte aligned only
            v = L.lift_variant_describe(op, vid)
            runs = vid if (v["stages"] == 0 and v["vw"] == 1) else 0   # else the guarded form
            exp, _ = expected_bits(L, opname, runs, x, y)
            assert got == exp
    got, _ = reduce_gpu(L, "asum", 14, x, offset=3)
    assert abs(float(got) - ref_a) <= blas.tolerance(n, blas.asum_terms(x))
    got, _ = reduce_gpu(L, "dot", 14, x, y, offset=2)
    assert abs(float(got) - ref_d) <= blas.tolerance(n, blas.dot_terms(x, y))


def test_reduce_edge_cases(L):
    r = torch.full((1,), 5.0, device="cuda")
    x = torch.zeros(8, device="cuda")
    for vid in (0, 14, 22, 29, 34):
        L.lift_asum_v(vid, x, 0, r)
        assert r.item() == 0.0
        L.lift_dot_v(vid, x, x, 0, r)
        assert r.item() == 0.0
    for n in (1, 31, 32, 255, 256, 257, 4095, 4096, 4097, (1 << 20) + 1):
        v = np.arange(n, dtype=np.float32) % 7 - 3
        got, _ = reduce_gpu(L, "asum", 14, v)
        assert float(got) == float(np.abs(v.astype(np.float64)).sum())
    # NaN and Inf propagate
    v = np.ones(10000, np.float32)
    v[1234] = np.nan
    assert np.isnan(reduce_gpu(L, "asum", 14, v)[0])
    v[1234] = np.inf
    assert reduce_gpu(L, "asum", 14, v)[0] == np.inf
    v[1234] = -np.inf
    assert reduce_gpu(L, "dot", 14, v, np.ones_like(v))[0] == -np.inf


def test_reduce_closed_forms(L):
    # asum of x_i = i/n is (n-1)/2; dot of constant vectors 0.5, 3 is 1.5 n
    n = 1 << 20
    x = (np.arange(n) / n).astype(np.float32)
    for vid in range(L.lift_variant_count(L.OP_ASUM)):
        got, got64 = reduce_gpu(L, "asum", vid, x)
        assert abs(got64 - (n - 1) / 2) <= blas.tolerance(n, (n - 1) / 2)
    c = np.full(n, 0.5, np.float32)
    for vid in range(L.lift_variant_count(L.OP_DOT)):
        got, got64 = reduce_gpu(L, "dot", vid, c, np.full(n, 3.0, np.float32))
        assert got64 == 1.5 * n     # every partial sum is an exact multiple of 1.5


# ---------------------------------------------------------------------------
# scal
# ---------------------------------------------------------------------------
def test_scal_all_variants_bit_exact_full_size(L, dot_case):
    x, _, alpha, _, _ = dot_case
    exp = blas.scal(alpha, x.astype(np.float64)).astype(np.float32).view(np.uint32)
    xd = dev(x)
    out = torch.empty_like(xd)
    for vid in range(L.lift_variant_count(L.OP_SCAL)):
        out.fill_(np.nan)
        L.lift_scal_v(vid, x.size, alpha, xd, out)
        got = out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, exp), L.lift_variant_describe(L.OP_SCAL, vid)["name"]


@pytest.mark.parametrize("n", [1, 3, 1023, 4097, 100003])
def test_scal_ragged_in_place_and_misaligned(L, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    x[0] = 1e-40                                       # subnormal: no flush to zero
    exp = (x.astype(np.float64) * 1.5).astype(np.float32).view(np.uint32)
    for vid in range(L.lift_variant_count(L.OP_SCAL)):
        buf = torch.zeros(n + 16, device="cuda")
        buf[:n] = dev(x)
        L.lift_scal_v(vid, n, 1.5, buf, buf)           # in place
        assert np.array_equal(buf[:n].cpu().numpy().view(np.uint32), exp)
        assert torch.all(buf[n:] == 0)                 # nothing written past n
        src = torch.zeros(n + 16, device="cuda")
        src[1:n + 1] = dev(x)
        dst = torch.zeros(n + 16, device="cuda")
        L.lift_scal_v(vid, n, 1.5, src.data_ptr() + 4, dst.data_ptr() + 12)
        assert np.array_equal(dst[3:n + 3].cpu().numpy().view(np.uint32), exp)
        assert torch.all(dst[:3] == 0) and torch.all(dst[n + 3:] == 0)


# ---------------------------------------------------------------------------
# gemv
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(8192, 8192), (65536, 1024)])
def test_gemv_all_variants_full_size_sampled_rows(L, shape):
    M, N = shape
    A, x, y, alpha, beta = synth.gemv(M, N)
    alpha, beta = float(alpha), float(beta)
    rows = np.sort(np.random.default_rng(5).choice(M, 96, replace=False))
    ref = blas.gemv(A[rows].astype(np.float64), x.astype(np.float64), y[rows].astype(np.float64),
                    alpha, beta)
    tol = blas.tolerance(N, 1.0) * blas.gemv_row_terms(A[rows], x, y[rows], alpha, beta)
    Ad, xd, y0 = dev(A), dev(x), dev(y)
    yd = torch.empty_like(y0)
    for vid in range(L.lift_variant_count(L.OP_GEMV)):
        yd.copy_(y0)
        L.lift_gemv_v(vid, M, N, alpha, Ad, N, xd, beta, yd)
        got = yd.cpu().numpy()[rows]
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (L.lift_variant_describe(L.OP_GEMV, vid)["name"], np.flatnonzero(bad)[:5])


@pytest.mark.parametrize("M,N", [(1, 1), (7, 33), (40, 257), (129, 1000), (33, 4100), (5, 8192),
                                 (3, 50000), (2, 300004), (9, 512), (40, 1280), (37, 2304)])
def test_gemv_bit_exact_to_expression(L, M, N):
    rng = np.random.default_rng(M * N)
    A = rng.standard_normal((M, N)).astype(np.float32)
    x = rng.standard_normal(N).astype(np.float32)
    y = rng.standard_normal(M).astype(np.float32)
    for vid in range(L.lift_variant_count(L.OP_GEMV)):
        v = L.lift_variant_describe(L.OP_GEMV, vid)
        # rows whose pitch (lda * 4 bytes) is not a multiple of the vector
        # load run the 4-byte form (variant 0)
        ok = (4 * N) % (4 * v["vw"]) == 0 and not (v["tree"] == 3 and N % 256 != 0)
        runs = v if ok else L.lift_variant_describe(L.OP_GEMV, 0)
        if runs["name"].startswith("gemv_split_"):
            seg, S = L.lift_gemv_segments(runs["id"], M, N)
            ze = ll.gemv_split_z_variant(M, N, 1.25, runs["vw"], runs["threads"], seg, S)
        else:
            ze = ll.gemv_z_variant(M, N, 1.25, runs["vw"], runs["lanes"], 1)
        for beta in (0.5, 0.0):
            z = evaluate(ze, A, mode="f32", env={"x": x})
            if beta != 0:
                exp = evaluate(C(Map(add), Zip()), (z, evaluate(Map(mult_by(beta)), y, mode="f32")),
                               mode="f32")
            else:
                exp = z
            yd = dev(y)
            L.lift_gemv_v(vid, M, N, 1.25, dev(A), N, dev(x), beta, yd)
            assert np.array_equal(yd.cpu().numpy(), exp.astype(np.float32)), (v["name"], beta)


def test_gemv_edge_cases(L):
    M, N, lda = 37, 70, 75
    rng = np.random.default_rng(9)
    A = rng.standard_normal((M, lda)).astype(np.float32)
    A[:, N:] = np.nan                                   # padding columns are never read
    x = rng.standard_normal(N).astype(np.float32)
    ref = blas.gemv(A[:, :N].astype(np.float64), x.astype(np.float64), np.zeros(M), 2.0, 0.0)
    for vid in range(L.lift_variant_count(L.OP_GEMV)):
        yd = torch.full((M,), float("nan"), device="cuda")   # beta = 0: y is not read
        L.lift_gemv_v(vid, M, N, 2.0, dev(A), lda, dev(x), 0.0, yd)
        got = yd.cpu().numpy()
        tol = blas.tolerance(N, 1.0) * blas.gemv_row_terms(A[:, :N], x, np.zeros(M), 2.0, 0.0)
        assert np.all(np.abs(got - ref) <= tol)
    yd = dev(np.arange(5, dtype=np.float32))
    L.lift_gemv(5, 0, 3.0, 0, 0, 0, 0.5, yd)               # N = 0: y <- beta * y
    assert yd.cpu().numpy().tolist() == [0.0, 0.5, 1.0, 1.5, 2.0]
    L.lift_gemv(0, 10, 1.0, 0, 10, 0, 1.0, 0)              # M = 0: nothing to do
    # closed form: A = 1, x = 1 -> y = alpha * N + beta * y
    A1 = torch.ones((64, 300), device="cuda")
    yd = dev(np.arange(64, dtype=np.float32))
    L.lift_gemv(64, 300, 2.0, A1, 300, torch.ones(300, device="cuda"), 0.5, yd)
    assert yd.cpu().numpy().tolist() == (2.0 * 300 + 0.5 * np.arange(64)).tolist()
