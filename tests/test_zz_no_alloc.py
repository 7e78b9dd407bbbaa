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


def test_noalloc_asum_misaligned_and_empty_inputs():
    """x may be any 4-byte aligned pointer, as for lift_asum: offsets of 1, 2
    and 3 floats go to the 4-byte-load form, which folds the same elements
    in the same order, so its result equals the aligned call's bit for bit
    and the oracle's within the parity bound.  n == 0 writes exactly 0."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    n = (1 << 21) + 4097                                  # ragged: a partial last tile
    x = synth.asum_small(n, seed=7)
    aligned = torch.from_numpy(x).cuda()
    ref = torch.full((1,), -1.0, device="cuda")
    lift.lift_asum_noalloc(aligned, n, ref)
    tol = blas.tolerance(n, blas.asum_terms(x))
    for off in (1, 2, 3):
        buf = torch.full((n + 8,), float("nan"), device="cuda")
        view = buf[off:off + n]
        view.copy_(aligned)
        assert view.data_ptr() % 16 != 0
        got = torch.full((1,), -1.0, device="cuda")
        lift.lift_asum_noalloc(view, n, got)
        torch.cuda.synchronize()
        assert float(got) == float(ref), off
        assert abs(float(got) - blas.asum(x.astype(np.float64))) <= tol
    zero = torch.full((1,), -1.0, device="cuda")
    lift.lift_asum_noalloc(aligned, 0, zero)
    torch.cuda.synchronize()
    assert float(zero) == 0.0
