"""Guard bands (the stand-in for a memory sanitizer): every output is written
into the middle of a buffer whose surrounding words hold a sentinel, and every
variant of every op that writes must leave the sentinels untouched -- with
ragged sizes, unaligned lengths and misaligned starts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
PAD = 64
SENT = -7.25                     # not a value any of the ops below can write


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


def guarded(n, off=0, fill=0.5):
    """(buffer, view): view has n elements starting off floats after PAD."""
    b = torch.full((n + 2 * PAD + off,), SENT, device="cuda")
    v = b[PAD + off:PAD + off + n]
    v.fill_(fill)
    return b, v


def intact(b, n, off=0):
    h = b.cpu().numpy()
    return np.all(h[:PAD + off] == SENT) and np.all(h[PAD + off + n:] == SENT)


def vec(n, seed):
    return torch.from_numpy(np.random.default_rng(seed).uniform(1, 2, n).astype(np.float32)).cuda()


@pytest.mark.parametrize("n,off", [(1, 0), (4099, 1), (262147, 3)])
def test_vector_outputs(L, n, off):
    x = vec(n, 1)
    for vid in range(L.lift_variant_count(L.OP_SCAL)):
        b, y = guarded(n, off)
        L.lift_scal_v(vid, n, 1.5, x, y)
        assert intact(b, n, off), ("scal", vid)
    for vid in range(L.lift_variant_count(L.OP_AXPY)):
        b, y = guarded(n, off)
        L.lift_axpy_v(vid, n, 1.5, x, y)
        assert intact(b, n, off), ("axpy", vid)
    for vid in range(L.lift_variant_count(L.OP_BLACKSCHOLES)):
        bc, c = guarded(n, off)
        bp, p = guarded(n, off)
        L.lift_blackscholes_v(vid, n, x * 20, 20.0, 0.02, 0.3, 1.0, c, p)
        assert intact(bc, n, off) and intact(bp, n, off), ("blackscholes", vid)


@pytest.mark.parametrize("M,N,off", [(1, 1, 0), (37, 1030, 1), (3000, 64, 2), (5, 70000, 0),
                                     (37, 1280, 0), (11, 512, 0)])
def test_matrix_outputs(L, M, N, off):
    A = vec(M * N, 2)
    for op, rows, cols, call in ((L.OP_GEMV, M, N, L.lift_gemv_v), (L.OP_GEMV_T, N, M, L.lift_gemv_t_v)):
        x = vec(cols, 3)
        for vid in range(L.lift_variant_count(op)):
            b, y = guarded(rows, off)
            call(vid, M, N, 1.0, A, N, x, 0.5, y)
            assert intact(b, rows, off), (op, L.lift_variant_describe(op, vid)["name"])


def test_scalar_results(L):
    n = 100003
    x, y = vec(n, 4), vec(n, 5)
    for op in (L.OP_ASUM, L.OP_DOT, L.OP_NRM2, L.OP_SUM, L.OP_ASUM_COMP, L.OP_DOT_COMP):
        for vid in range(L.lift_variant_count(op)):
            b, r = guarded(1)
            if op == L.OP_ASUM:
                L.lift_asum_v(vid, x, n, r)
            elif op == L.OP_DOT:
                L.lift_dot_v(vid, x, y, n, r)
            elif op == L.OP_NRM2:
                L.lift_nrm2_v(vid, x, n, r)
            elif op == L.OP_SUM:
                L.lift_sum_v(vid, x, n, r)
            elif op == L.OP_ASUM_COMP:
                L.lift_asum_comp_v(vid, x, n, r)
            else:
                L.lift_dot_comp_v(vid, x, y, n, r)
            assert intact(b, 1), (op, vid)
