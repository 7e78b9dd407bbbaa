"""LIFT_POLICY_MLP_TUNE on the host: the weights file's trained range
("box") is parsed and checked, lift_pick never times (it reports the
learned pick, or a cached winner), and nothing is timed before a call."""
import os

import pytest

from paper_1502_02389_gb300 import build, costmodel, lift


@pytest.fixture(scope="module")
def L():
    build.build()
    yield lift
    lift.lift_set_policy(lift.POLICY_FIXED)


def test_tune_policy_loads_and_picks_like_the_model(L):
    shapes = [(L.OP_ASUM, 1 << 20, 0, 0), (L.OP_DOT, 1 << 29, 0, 0),
              (L.OP_GEMV, 8192 * 8192, 8192, 8192), (L.OP_GEMV_T, 1 << 29, 1 << 14, 1 << 15)]
    L.lift_set_policy(L.POLICY_MLP, costmodel.WEIGHTS)
    plain = [L.lift_pick(*s) for s in shapes]
    L.lift_set_policy(L.POLICY_MLP_TUNE, costmodel.WEIGHTS)
    assert [L.lift_pick(*s) for s in shapes] == plain
    assert L.lift_tune_stats() == (0, 0)


def test_box_is_the_trained_range(L):
    # every op of the committed model has a box, and the benchmark shapes
    # lie inside it (so the fallback never times them)
    text = open(costmodel.WEIGHTS).read().split("box", 1)[1].split()
    count = int(text[0])
    rows = [text[1 + 7 * i: 8 + 7 * i] for i in range(count)]
    assert count == L.NUM_OPS and sorted(int(r[0]) for r in rows) == list(range(L.NUM_OPS))
    lo, hi = {int(r[0]): float(r[1]) for r in rows}, {int(r[0]): float(r[2]) for r in rows}
    for op in (L.OP_DOT, L.OP_SCAL):
        assert lo[op] <= 26 <= hi[op]


@pytest.mark.parametrize("tail, ok", [("box 1\n0 8 28 0 0 0 0\n", True),
                                      ("box 1\n0 8 28 0 0\n", False),
                                      ("box 1\n99 8 28 0 0 0 0\n", False),
                                      ("boxes 1\n", False)])
def test_box_parsing(L, tmp_path, tail, ok):
    body = open(costmodel.WEIGHTS).read().split("box", 1)[0]
    p = tmp_path / "w.txt"
    p.write_text(body + tail)
    if ok:
        L.lift_set_policy(L.POLICY_MLP_TUNE, str(p))
    else:
        with pytest.raises(L.LiftError) as e:
            L.lift_set_policy(L.POLICY_MLP_TUNE, str(p))
        assert e.value.status == L.ERR_INVALID_ARG
    L.lift_set_policy(L.POLICY_FIXED)
