"""Compensated fp32 asum and dot against the correctly rounded exact sums:
the full-size workload, an ill-conditioned dot whose cancellation defeats the
plain fold's bound, ragged and misaligned inputs, edge cases."""
import math

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


def per_pair(L, op, vid, n):
    """Terms per (sum, compensation) pair of a variant for n elements."""
    v = L.lift_variant_describe(op, vid)
    g = L.lift_variant_grid(op, vid, n)
    return max(1, math.ceil(n / (g * v["threads"] * v["vw"])))


def run(L, op, vid, x, y=None):
    r = torch.empty(1, device="cuda")
    r64 = torch.empty(1, dtype=torch.float64, device="cuda")
    if op == L.OP_ASUM_COMP:
        L.lift_asum_comp_v(vid, x, x.numel(), r, r64)
    else:
        L.lift_dot_comp_v(vid, x, y, x.numel(), r, r64)
    return float(r.item()), float(r64.item())


def test_full_size(L):
    n = 1 << 26
    xh, yh, _ = synth.dot_scal(n)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    exact_d = blas.dot_exact(xh, yh)
    terms_d = float(np.sum(np.abs(xh.astype(np.float64) * yh)))
    exact_a = blas.asum_exact(xh)
    for op, exact, terms in ((L.OP_DOT_COMP, exact_d, terms_d), (L.OP_ASUM_COMP, exact_a, exact_a)):
        for vid in range(L.lift_variant_count(op)):
            got, got64 = run(L, op, vid, x, y)
            tol = blas.compensated_tolerance(exact, terms, per_pair(L, op, vid, n))
            name = L.lift_variant_describe(op, vid)["name"]
            assert abs(got - exact) <= tol, (name, got, exact, tol)
            assert got == np.float32(got64), name


def test_ill_conditioned_dot(L):
    # y cancels x on the second half up to a 2^-12 relative perturbation:
    # |dot| is about 1e-4 of sum |x y|
    n = 1 << 22
    g = np.random.default_rng(8)
    a = g.standard_normal(n // 2).astype(np.float32)
    xh = np.concatenate([a, a])
    pert = (a * (1 + g.uniform(-2 ** -12, 2 ** -12, n // 2))).astype(np.float32)
    yh = np.concatenate([a, -pert])
    exact = blas.dot_exact(xh, yh)
    terms = float(np.sum(np.abs(xh.astype(np.float64) * yh)))
    assert abs(exact) < 1e-3 * terms
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    for vid in range(L.lift_variant_count(L.OP_DOT_COMP)):
        got, _ = run(L, L.OP_DOT_COMP, vid, x, y)
        tol = blas.compensated_tolerance(exact, terms, per_pair(L, L.OP_DOT_COMP, vid, n))
        assert abs(got - exact) <= tol, (vid, got, exact, tol)
    # the plain fold meets only its own, much wider bound
    r = torch.empty(1, device="cuda")
    L.lift_dot(x, y, n, r)
    assert abs(r.item() - exact) <= blas.tolerance(n, terms)


@pytest.mark.parametrize("n", [0, 1, 7, 4099, 1000003])
def test_ragged_and_misaligned(L, n):
    g = np.random.default_rng(n)
    xh = g.standard_normal(n + 1).astype(np.float32)
    yh = g.standard_normal(n + 1).astype(np.float32)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    for off in (0, 1):                          # offset 1: only 4-byte aligned
        xs, ys = xh[off:off + n], yh[off:off + n]
        for op in (L.OP_ASUM_COMP, L.OP_DOT_COMP):
            exact = blas.asum_exact(xs) if op == L.OP_ASUM_COMP else blas.dot_exact(xs, ys)
            terms = blas.asum_exact(xs) if op == L.OP_ASUM_COMP else \
                float(np.sum(np.abs(xs.astype(np.float64) * ys)))
            for vid in range(L.lift_variant_count(op)):
                r = torch.empty(1, device="cuda")
                if op == L.OP_ASUM_COMP:
                    L.lift_asum_comp_v(vid, x[off:], n, r)
                else:
                    L.lift_dot_comp_v(vid, x[off:], y[off:], n, r)
                tol = blas.compensated_tolerance(exact, terms, max(1, n))
                assert abs(r.item() - exact) <= tol, (op, vid, off)
