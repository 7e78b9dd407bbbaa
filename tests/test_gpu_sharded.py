"""Sharded asum / dot on one GPU: uneven shards reduced with
lift_asum_partial / lift_dot_partial, combined with lift_combine_partials,
against the whole-vector oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas
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


def test_shards_combine_to_the_whole(L):
    n = (1 << 24) + 77
    xh, yh, _ = synth.dot_scal(n)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    cuts = [0, 1000, 5_000_003, 9_999_999, n]           # uneven, unaligned shards
    pa = torch.zeros(len(cuts) - 1, dtype=torch.float64, device="cuda")
    pd = torch.zeros_like(pa)
    for i in range(len(cuts) - 1):
        a, b = cuts[i], cuts[i + 1]
        L.lift_asum_partial(x[a:b], b - a, pa[i:i + 1])
        L.lift_dot_partial(x[a:b], y[a:b], b - a, pd[i:i + 1])
    ra, _ = L.lift_combine_partials(pa.cpu().numpy().tolist())
    rd, _ = L.lift_combine_partials(pd.cpu().numpy().tolist())
    assert abs(ra - blas.asum(xh)) <= blas.tolerance(n, blas.asum_terms(xh))
    assert abs(rd - blas.dot(xh, yh)) <= blas.tolerance(n, blas.dot_terms(xh, yh))
    # one shard: the partial is the FP64 value the plain call rounds
    r = torch.empty(1, device="cuda")
    L.lift_asum(x, n, r)
    L.lift_asum_partial(x, n, pa[0:1])
    assert r.item() == np.float32(pa[0].item())
