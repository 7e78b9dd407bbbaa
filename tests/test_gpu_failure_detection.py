"""The device-side timeout path, exercised without a fault: a wait that
nothing satisfies gives up after its poll limit, the status word reports
LIFT_ERR_TIMEOUT, reading it clears it, and the context stays usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    return lift


def test_wait_gives_up_and_reports(L):
    assert L.lift_read_status(1) == 0
    t = time.perf_counter()
    L.lift_wait_probe(256)
    torch.cuda.synchronize()
    assert time.perf_counter() - t < 5.0
    assert L.lift_read_status(1) == L.ERR_TIMEOUT       # reported ...
    assert L.lift_read_status(1) == 0                   # ... and cleared by the read
    # the context is still usable: a staged (bulk-copy) variant computes correctly
    x = np.random.default_rng(0).standard_normal(1 << 20).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    r = torch.empty(1, device="cuda")
    vid = [v["id"] for v in L.variants(L.OP_ASUM) if v["stages"] > 0][0]
    L.lift_asum_v(vid, xd, x.size, r)
    assert abs(r.item() - blas.asum(x)) <= blas.tolerance(x.size, blas.asum_terms(x))
    assert L.lift_read_status(1) == 0


def test_probe_arguments(L):
    with pytest.raises(L.LiftError):
        L.lift_wait_probe(0)
    with pytest.raises(L.LiftError):
        L.lift_wait_probe((1 << 22) + 1)
