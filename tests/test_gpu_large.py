"""Sizes past 2^31 elements (64-bit indexing in every kernel), checked through
values that are exact at any size: a few nonzero markers, one of them past
index 2^31, in a vector of zeros (every partial sum is a small integer); gemv
and gemv-T with A = 1, x = 1, whose row and column sums are integers below
2^24, so y = alpha*N + beta*y exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BIG = (1 << 31) + 4099          # elements: 8.6 GB of fp32


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


def test_asum_sum_nrm2_past_2_31(L):
    x = torch.zeros(BIG, device="cuda")
    for i, v in ((5, -4.0), ((1 << 31) + 7, 2.0), (BIG - 1, 1.0)):
        x[i] = v
    r = torch.empty(1, device="cuda")
    r64 = torch.empty(1, dtype=torch.float64, device="cuda")
    for vid in range(L.lift_variant_count(L.OP_ASUM)):
        L.lift_asum_v(vid, x, BIG, r, r64)
        assert r64.item() == 7.0 and r.item() == 7.0, L.lift_variant_describe(L.OP_ASUM, vid)["name"]
    L.lift_sum(x, BIG, r)
    assert r.item() == -1.0
    L.lift_nrm2(x, BIG, r)
    assert r.item() == float(np.float32(np.sqrt(21.0)))
    L.lift_asum_comp(x, BIG, r, r64)
    assert r64.item() == 7.0
    L.lift_dot(x, x, BIG, r)
    assert r.item() == 21.0
    del x
    torch.cuda.empty_cache()


def test_gemv_and_gemv_t_past_2_31(L):
    M, N = 40000, 53696             # M*N = 2,147,840,000 > 2^31
    A = torch.ones((M, N), device="cuda")
    for op, rows, cols, call in ((L.OP_GEMV, M, N, L.lift_gemv_v), (L.OP_GEMV_T, N, M, L.lift_gemv_t_v)):
        x = torch.ones(cols, device="cuda")
        y0 = torch.arange(rows, dtype=torch.float32, device="cuda")
        want = (2.0 * cols + 0.5 * y0).cpu().numpy()
        for vid in range(L.lift_variant_count(op)):
            y = y0.clone()
            call(vid, M, N, 2.0, A, N, x, 0.5, y)
            assert np.array_equal(y.cpu().numpy(), want), (op, L.lift_variant_describe(op, vid)["name"])
    del A
    torch.cuda.empty_cache()
