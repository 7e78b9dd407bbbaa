"""lift_asum_noalloc, the allocation-free asum.

It serves callers that cannot let a library allocate device memory: a
process whose device memory is owned by its own pool allocator under a
fixed budget, or a latency-critical loop that cannot afford the
device-wide synchronisation of cudaFree.  Its scratch is a fixed array in
the library's device image, shared by every call, so this test makes two
calls in a row (different sizes, the second one ragged) and checks each
result against lift_asum's, which uses the cudaMalloc'ed workspace, within
the parity tolerance.  It needs no other test to have run first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas
from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_asum_matches_lift_asum_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    xs = [synth.asum_small(1 << 20, seed=0), synth.asum_small((1 << 22) + 12345, seed=5)]
    xd = [torch.from_numpy(x).cuda() for x in xs]
    got = torch.full((2,), -1.0, device="cuda")
    for i, (x, d) in enumerate(zip(xs, xd)):          # no lift_init needed
        lift.lift_asum_noalloc(d, x.size, got[i:i + 1])
    torch.cuda.synchronize()
    lift.lift_init(0)
    ref = torch.full((2,), -1.0, device="cuda")
    for i, (x, d) in enumerate(zip(xs, xd)):
        lift.lift_asum(d, x.size, ref[i:i + 1])
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        tol = blas.tolerance(x.size, blas.asum_terms(x))
        assert abs(float(got[i]) - float(ref[i])) <= tol
        assert abs(float(got[i]) - blas.asum(x.astype(np.float64))) <= tol
    with pytest.raises(lift.LiftError) as e:
        lift.lift_asum_noalloc(xd[0], -1, got[:1])
    assert e.value.status == lift.ERR_INVALID_ARG
