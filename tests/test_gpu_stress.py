"""Long per-lane chains under inputs that make a plain fp32 fold's error grow
with its length.

Same-sign constant terms (1.3, 0.6: every add of a plain chain loses about
half an ulp of the running sum in the same direction, so its relative error
grows linearly -- 73u after 432 terms) and same-sign decreasing terms, on
every variant of the long-chain families:

* asum / sum / dot at n = 2^26 (the grids leave 54-108 tiles per lane);
* gemv-T at 65536 x 1024 (column blocks of 100+ rows per thread);
* gemv on 1024 x 65536 (rows of 512 vectors per lane: a plain chain would
  err by about 70u against a parity bound of 4u * 16 = 64u).

Each result must lie within the parity bound 4u * ceil(log2 n) * sum|t| and
within its variant's structural bound: the terms a lane folds plainly
before a compensated add, plus 2 for the compensation, plus the adds on the
longest path of the lane sum, the trees and the epilogue, times u * sum|t|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


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


def _tree_depth(threads: int, cluster: int) -> int:
    # warp halving tree, the second warp tree over the warp results, the
    # rank-ordered cluster sum
    return 5 + (5 if threads > 32 else 0) + (cluster - 1)


def reduction_bound(v) -> float:
    """Adds on the longest path of a reduction variant's value, per unit of
    u * sum|t| (same-sign terms): the tile's J vectors folded plainly in a
    lane, the lane sum, the compensated tile sum (2), the trees, the final
    rounding of the FP64 combine (1)."""
    J = v["tile"] // (v["vw"] * v["threads"])
    return J + (v["vw"] - 1) + 2 + _tree_depth(v["threads"], v["cluster"]) + 1


def _data(n, kind, seed_scale=1.3):
    if kind == "const":
        return np.full(n, np.float32(seed_scale), np.float32)
    i = np.arange(n, dtype=np.float64)
    return (seed_scale * (2.0 - i / n)).astype(np.float32)      # same sign, decreasing


@pytest.mark.parametrize("kind", ["const", "decreasing"])
def test_reductions_long_chains(L, kind):
    n = 1 << 26
    x = _data(n, kind, 1.3)
    y = _data(n, kind, 0.6)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ref = {"asum": blas.asum(x), "sum": blas.sum_(x), "dot": blas.dot(x, y)}
    terms = {"asum": blas.asum_terms(x), "sum": blas.asum_terms(x), "dot": blas.dot_terms(x, y)}
    r = torch.empty(1, device="cuda")
    worst = {}
    for name, op, call in (("asum", L.OP_ASUM, lambda v: L.lift_asum_v(v, xd, n, r)),
                           ("sum", L.OP_SUM, lambda v: L.lift_sum_v(v, xd, n, r)),
                           ("dot", L.OP_DOT, lambda v: L.lift_dot_v(v, xd, yd, n, r))):
        tol = blas.tolerance(n, terms[name])
        for v in L.variants(op):
            call(v["id"])
            torch.cuda.synchronize()
            err = abs(float(r.item()) - ref[name])
            bound = reduction_bound(v) * U * terms[name]
            assert err <= tol, (v["name"], err / (U * terms[name]))
            assert err <= bound, (v["name"], err / (U * terms[name]), reduction_bound(v))
            worst[name] = max(worst.get(name, 0.0), err / (U * terms[name]))
    print(kind, {k: round(w, 3) for k, w in worst.items()}, "(error / (u sum|t|))")


@pytest.mark.parametrize("kind", ["const", "decreasing"])
def test_gemv_t_long_column_chains(L, kind):
    M, N = 65536, 1024
    col = _data(M, kind, 1.3)                       # A_ij = col_i for every column j
    A = np.repeat(col[:, None], N, axis=1)
    x = np.ones(M, np.float32)
    Ad, xd = torch.from_numpy(A).cuda(), torch.from_numpy(x).cuda()
    cols = np.array([0, 1, 511, 1023])
    ref = blas.gemv_t(A[:, cols].astype(np.float64), x.astype(np.float64), np.zeros(cols.size), 1.0, 0.0)
    terms = float(np.sum(np.abs(col.astype(np.float64))))
    tol = blas.tolerance(M, terms)
    worst = 0.0
    for v in L.variants(L.OP_GEMV_T):
        yd = torch.zeros(N, device="cuda")
        L.lift_gemv_t_v(v["id"], M, N, 1.0, Ad, N, xd, 0.0, yd)
        got = yd.cpu().numpy()[cols].astype(np.float64)
        err = float(np.max(np.abs(got - ref)))
        # 32 rows folded plainly, compensation (2), the combine's longest
        # path (two pass: compensated lane fold 2 + halving tree 5; cluster:
        # CL - 1 + 2; one pass: 2), the epilogue product (1)
        combine = 7 if v["passes"] == 2 else (v["cluster"] - 1 + 2 if v["cluster"] > 1 else 2)
        bound = (32 + 2 + combine + 1) * U * terms
        assert err <= tol, (v["name"], err / (U * terms))
        assert err <= bound, (v["name"], err / (U * terms))
        worst = max(worst, err / (U * terms))
    print(kind, "gemv-T worst", round(worst, 3), "(error / (u sum|t|))")


@pytest.mark.parametrize("kind", ["const", "decreasing"])
def test_gemv_long_rows(L, kind):
    M, N = 1024, 65536
    row = _data(N, kind, 0.6)                       # every row the same
    A = np.repeat(row[None, :], M, axis=0)
    x = np.ones(N, np.float32)
    Ad, xd = torch.from_numpy(A).cuda(), torch.from_numpy(x).cuda()
    ref = blas.gemv(A[:2].astype(np.float64), x.astype(np.float64), np.zeros(2), 1.0, 0.0)[0]
    terms = float(np.sum(np.abs(row.astype(np.float64))))
    tol = blas.tolerance(N, terms)
    worst = 0.0
    for v in L.variants(L.OP_GEMV):
        yd = torch.zeros(M, device="cuda")
        L.lift_gemv_v(v["id"], M, N, 1.0, Ad, N, xd, 0.0, yd)
        got = yd.cpu().numpy().astype(np.float64)
        err = float(np.max(np.abs(got - ref)))
        # a lane's group of 8 vectors (8 terms per vector lane), the lane sum
        # (vw - 1), compensation (2), the trees (a warp tree; a CTA's second
        # tree and the compensated segment combine for split rows), the
        # epilogue product (1)
        trees = 5 + (5 + 2 + 5 if v["name"].startswith("gemv_split") else 0)
        bound = (8 + (v["vw"] - 1) + 2 + trees + 1) * U * terms
        assert err <= tol, (v["name"], err / (U * terms))
        assert err <= bound, (v["name"], err / (U * terms))
        worst = max(worst, err / (U * terms))
    print(kind, "gemv worst", round(worst, 3), "(error / (u sum|t|))")
