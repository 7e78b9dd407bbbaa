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


def test_memoised_picks_follow_reloaded_weights(L, tmp_path):
    # picks are memoised per call shape; loading other weights must not
    # return the memo of the previous ones
    lines = open(costmodel.WEIGHTS).read().split("\n")
    head = lines[0].split()
    d_in, h1, h2, V = (int(v) for v in head[2:6])
    off = [int(v) for v in lines[1].split()[2:]]
    params = [float(v) for v in lines[2].split()]
    n_before_b3 = d_in * h1 + h1 + h1 * h2 + h2 + h2 * V
    for shape in ((L.OP_DOT, 1 << 26, 0, 0), (L.OP_ASUM, 1 << 22, 0, 0)):
        op = shape[0]
        L.lift_set_policy(L.POLICY_MLP, costmodel.WEIGHTS)
        first = L.lift_pick(*shape)
        assert L.lift_pick(*shape) == first                 # memoised, same answer
        other = 0 if first != 0 else 1
        p2 = list(params)
        p2[n_before_b3 + off[op] + other] -= 1000.0         # make `other` predicted fastest
        lines2 = list(lines)
        lines2[2] = " ".join(f"{v:.9g}" for v in p2)
        w2 = tmp_path / f"w{op}.txt"
        w2.write_text("\n".join(lines2))
        L.lift_set_policy(L.POLICY_MLP, str(w2))
        assert L.lift_pick(*shape) == other
        L.lift_set_policy(L.POLICY_MLP, costmodel.WEIGHTS)
        assert L.lift_pick(*shape) == first
    L.lift_set_policy(L.POLICY_FIXED)
