"""Autotuner: timing database, resume, and the TABLE policy built from it."""
import json
import math

import pytest

from paper_1502_02389_gb300 import build, lift, tune


@pytest.fixture(scope="module")
def L():
    build.build()
    lift.lib()
    return lift


def fake_records():
    recs = []
    for op, n, best in ((lift.OP_DOT, 1 << 10, 3), (lift.OP_DOT, 1 << 26, 14), (lift.OP_ASUM, 1 << 20, 7)):
        for v in range(lift.lift_variant_count(op)):
            recs.append({"device": "d", "op": op, "n": n, "M": 0, "N": 0, "variant": v,
                         "ms": 1.0 if v == best else 2.0 + v})
    recs.append({"device": "d", "op": lift.OP_GEMV, "n": 8192 * 8192, "M": 8192, "N": 8192,
                 "variant": 2, "ms": 1.0})
    return recs


def test_table_policy_picks_nearest_measured_best(L, tmp_path):
    p = tmp_path / "table.txt"
    tune.write_table(fake_records(), str(p))
    L.lift_set_policy(L.POLICY_TABLE, str(p))
    try:
        assert L.lift_pick(L.OP_DOT, 1 << 11) == 3          # nearest: 2^10
        assert L.lift_pick(L.OP_DOT, 1 << 25) == 14         # nearest: 2^26
        assert L.lift_pick(L.OP_ASUM, 5) == 7
        assert L.lift_pick(L.OP_GEMV, 0, 8000, 8000) == 2
        L.lift_set_variant(L.OP_DOT, 5)                     # an override wins
        assert L.lift_pick(L.OP_DOT, 1 << 11) == 5
        L.lift_set_variant(L.OP_DOT, -1)
    finally:
        L.lift_set_policy(L.POLICY_FIXED)


def test_bad_table_is_rejected(L, tmp_path):
    p = tmp_path / "bad.txt"
    p.write_text("0 10 0 0 100000\n")
    with pytest.raises(L.LiftError):
        L.lift_set_policy(L.POLICY_TABLE, str(p))
    with pytest.raises(L.LiftError):
        L.lift_set_policy(L.POLICY_TABLE, str(tmp_path / "missing.txt"))


def test_op_bytes_and_shapes():
    assert tune.op_bytes(lift.OP_DOT, 100) == 800
    assert tune.op_bytes(lift.OP_GEMV, 0, 10, 20) == 4 * 200 + 80 + 80
    assert tune.op_bytes(lift.OP_DOT_FP8, 5000) == 2 * (5000 + 4 * 2)
    s = tune.random_shapes(300, seed=1)
    assert s == tune.random_shapes(300, seed=1)
    assert all(2 ** 8 - 1 <= n <= 2 ** 28 + 1 for op, n, M, N in s if op != lift.OP_GEMV)
    assert all(M * N == n and M * N <= 2 ** 28 for op, n, M, N in s if op == lift.OP_GEMV)
    assert {op for op, *_ in s} == set(tune.DEFAULT_SHAPE_OPS)
    t = tune.random_shapes(200, seed=2, ops=[lift.OP_GEMV_T, lift.OP_NRM2])
    assert all(M * N == n for op, n, M, N in t if op == lift.OP_GEMV_T)


@pytest.mark.gpu
def test_sweep_writes_and_resumes(L, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    db = str(tmp_path / "db.jsonl")
    shapes = [(L.OP_ASUM, 5000, 0, 0), (L.OP_SCAL, 70000, 0, 0), (L.OP_GEMV, 64 * 300, 64, 300),
              (L.OP_DOT_FP8, 9000, 0, 0)]
    recs = tune.sweep(shapes, db, reps=3, warmup=1)
    counts = sum(L.lift_variant_count(op) for op, *_ in shapes)
    assert len(recs) == counts
    assert all(r["ms"] > 0 and r["gbs"] > 0 for r in recs)
    assert len(tune.sweep(shapes, db, reps=3, warmup=1)) == 0      # resumed: nothing left
    assert len(tune.load_db(db)) == counts


def test_committed_cost_model_beats_the_method_without_it(L, tmp_path):
    """The weights under data/ (trained on the GPU from the committed sweep),
    loaded by the library's MLP policy, pick variants within 10 % of the
    exhaustive best on the held-out shapes, better than the best fixed
    variant per op."""
    import os
    from paper_1502_02389_gb300 import costmodel as cm
    tr = tune.load_csv(os.path.join(cm.DATA, "timings_gb300_train.csv"))
    ho = tune.load_csv(os.path.join(cm.DATA, "timings_gb300_heldout.csv"))
    res = cm.evaluate_policies(tr, ho, cm.WEIGHTS, str(tmp_path / "table.txt"))
    assert res["mlp"]["shapes"] >= 499
    assert res["mlp"]["geomean"] <= 1.10
    assert res["mlp"]["geomean"] < res["best_fixed"]["geomean"]
    assert res["mlp"]["geomean"] < res["table"]["geomean"]


def test_committed_cost_model_on_the_benchmark_shapes(L):
    """On the benchmark configurations (every op's workload shapes, timed with
    every variant) the learned pick is within 2 % of the exhaustive best."""
    import os
    from paper_1502_02389_gb300 import costmodel as cm
    wl = tune.load_csv(os.path.join(cm.DATA, "timings_gb300_workloads.csv"))
    L.lift_set_policy(L.POLICY_MLP, cm.WEIGHTS)
    try:
        r = cm.regrets(wl, lambda op, n, M, N: L.lift_pick(op, n, M, N))
    finally:
        L.lift_set_policy(L.POLICY_FIXED)
    assert len(r) >= 19 and r.max() <= 1.02
