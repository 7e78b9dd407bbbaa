"""gemv-T against the oracle: tolerance on the two workload shapes (sampled
columns), bit for bit against each variant's low-level expression, edge
cases."""
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


@pytest.mark.parametrize("shape", [(8192, 8192), (65536, 1024)])
def test_full_size_sampled_columns(L, shape):
    M, N = shape
    A, _, _, alpha, beta = synth.gemv(M, N)
    g = synth.generator(5)
    x = g.uniform(-1, 1, M).astype(np.float32)
    y = g.uniform(-1, 1, N).astype(np.float32)
    cols = np.sort(np.random.default_rng(6).choice(N, 64, replace=False))
    As = A[:, cols].astype(np.float64)
    ref = blas.gemv_t(As, x.astype(np.float64), y[cols].astype(np.float64), float(alpha), float(beta))
    terms = abs(float(alpha)) * (np.abs(As).T @ np.abs(x.astype(np.float64))) + \
        np.abs(float(beta) * y[cols].astype(np.float64))
    tol = blas.tolerance(M, 1.0) * terms
    Ad, xd = dev(A), dev(x)
    for vid in range(L.lift_variant_count(L.OP_GEMV_T)):
        yd = dev(y)
        L.lift_gemv_t_v(vid, M, N, float(alpha), Ad, N, xd, float(beta), yd)
        got = yd.cpu().numpy()[cols]
        assert np.all(np.abs(got - ref) <= tol), L.lift_variant_describe(L.OP_GEMV_T, vid)["name"]


@pytest.mark.parametrize("M,N", [(1, 1), (37, 9), (300, 1030), (5000, 64), (20000, 96)])
def test_bit_exact_to_expression(L, M, N):
    rng = np.random.default_rng(M + N)
    A = rng.standard_normal((M, N)).astype(np.float32)
    x = rng.standard_normal(M).astype(np.float32)
    y = rng.standard_normal(N).astype(np.float32)
    for vid in range(L.lift_variant_count(L.OP_GEMV_T)):
        # a pitch that is not a multiple of the vector width runs the
        # 4-byte-load variant 0 instead
        info = L.lift_variant_describe(L.OP_GEMV_T, vid)
        run = vid if N % info["vw"] == 0 else 0
        B, RB = L.lift_gemv_t_blocks(run, M, N)
        rinfo = L.lift_variant_describe(L.OP_GEMV_T, run)
        z = evaluate(ll.gemv_t_z_variant(M, N, 1.25, B, RB, rinfo["passes"], rinfo["cluster"]), A,
                     mode="f32", env={"x": x})
        for beta in (0.5, 0.0):
            exp = z if beta == 0 else evaluate(
                C(Map(add), Zip()), (z, evaluate(Map(mult_by(beta)), y, mode="f32")), mode="f32")
            yd = dev(y)
            L.lift_gemv_t_v(vid, M, N, 1.25, dev(A), N, dev(x), beta, yd)
            assert np.array_equal(yd.cpu().numpy(), exp.astype(np.float32)), (vid, beta)


def test_edge_cases(L):
    yd = dev(np.arange(6, dtype=np.float32))
    L.lift_gemv_t(0, 6, 2.0, 0, 6, 0, 0.5, yd)          # M = 0: y <- beta * y
    assert yd.cpu().numpy().tolist() == [0.0, 0.5, 1.0, 1.5, 2.0, 2.5]
    L.lift_gemv_t(5, 0, 1.0, 0, 0, 0, 1.0, 0)            # N = 0: nothing
    M, N, lda = 50, 30, 33                                # padded rows, unaligned pitch
    A = np.random.default_rng(1).standard_normal((M, lda)).astype(np.float32)
    A[:, N:] = np.nan
    x = np.ones(M, np.float32)
    yd = torch.full((N,), float("nan"), device="cuda")   # beta = 0: y not read
    L.lift_gemv_t(M, N, 1.0, dev(A), lda, dev(x), 0.0, yd)
    ref = A[:, :N].astype(np.float64).sum(axis=0)
    assert np.allclose(yd.cpu().numpy(), ref, rtol=0, atol=1e-4)


@pytest.mark.parametrize("M,N", [(300, 1028), (4099, 96)])
def test_padded_pitch_and_offsets(L, M, N):
    """Rows lda = N + 4 apart with NaN in the padding (the staged forms copy
    only the N floats of each row segment), and A, x 4 bytes off a 16-byte
    boundary (every vector variant runs its fallback then): bit for bit
    against each variant's expression on the unpadded matrix."""
    rng = np.random.default_rng(M * 7 + N)
    lda = N + 4
    A = rng.standard_normal((M, N)).astype(np.float32)
    Ap = np.full((M, lda), np.nan, np.float32)
    Ap[:, :N] = A
    x = rng.standard_normal(M).astype(np.float32)
    y = rng.standard_normal(N).astype(np.float32)
    for vid in range(L.lift_variant_count(L.OP_GEMV_T)):
        info = L.lift_variant_describe(L.OP_GEMV_T, vid)
        for offset in (0, 1):
            # the library's rule: A, x (and y) and the pitch aligned to the
            # variant's vectors (16 bytes for the staged copies, which also
            # need N % 4 == 0); otherwise the 4-byte-load variant 0 runs
            al = 16 if info["stages"] > 0 else 4 * info["vw"]
            ok = (offset == 0 or al <= 4) and (lda * 4) % al == 0 and \
                (info["stages"] == 0 or N % 4 == 0)
            run = vid if ok else 0
            B, RB = L.lift_gemv_t_blocks(run, M, N)
            rinfo = L.lift_variant_describe(L.OP_GEMV_T, run)
            z = evaluate(ll.gemv_t_z_variant(M, N, 0.75, B, RB, rinfo["passes"], rinfo["cluster"]), A,
                         mode="f32", env={"x": x})
            exp = evaluate(C(Map(add), Zip()), (z, evaluate(Map(mult_by(0.5)), y, mode="f32")),
                           mode="f32").astype(np.float32)
            Abuf = torch.zeros(M * lda + 8, device="cuda")
            Abuf[offset:offset + M * lda] = dev(Ap.reshape(-1))
            xbuf = torch.zeros(M + 8, device="cuda")
            xbuf[offset:offset + M] = dev(x)
            yd = dev(y)
            L.lift_gemv_t_v(vid, M, N, 0.75, Abuf.data_ptr() + 4 * offset, lda,
                            xbuf.data_ptr() + 4 * offset, 0.5, yd)
            assert np.array_equal(yd.cpu().numpy(), exp), (info["name"], offset)
