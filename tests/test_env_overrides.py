"""LIFT_POLICY / LIFT_VARIANT, read at the first lift_init (before any device
work, so this runs without a GPU): a forced variant and a policy show in
lift_pick; unknown names make lift_init fail with LIFT_ERR_INVALID_ARG."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import json, sys
sys.path.insert(0, %r)
from paper_1502_02389_gb300 import lift
rc = lift.lib().lift_init(0)
print(json.dumps({"rc": rc,
                  "dot": lift.lift_variant_describe(lift.OP_DOT, lift.lift_pick(lift.OP_DOT, 1 << 26))["name"],
                  "scal": lift.lift_variant_describe(lift.OP_SCAL, lift.lift_pick(lift.OP_SCAL, 1 << 26))["name"],
                  "asum_small": lift.lift_pick(lift.OP_ASUM, 1 << 12)}))
""" % ROOT


def probe(env):
    from paper_1502_02389_gb300 import build
    build.build()
    e = dict(os.environ)
    e.pop("LIFT_POLICY", None)
    e.pop("LIFT_VARIANT", None)
    e.update(env)
    out = subprocess.run([sys.executable, "-c", PROBE], env=e, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_forced_variants_and_policy():
    from paper_1502_02389_gb300 import lift
    base = probe({})
    r = probe({"LIFT_VARIANT": "dot_t1024_v1_ldg_p1,scal_t256_v1_ldg", "LIFT_POLICY": "mlp"})
    assert r["rc"] != lift.ERR_INVALID_ARG
    assert r["dot"] == "dot_t1024_v1_ldg_p1" and r["scal"] == "scal_t256_v1_ldg"
    assert base["dot"] != r["dot"]
    # the learned policy from the weights beside the library, as set_policy would
    lift.lift_set_policy(lift.POLICY_MLP, os.path.join(ROOT, "paper_1502_02389_gb300", "data",
                                                       "mlp_gb300.txt"))
    try:
        assert r["asum_small"] == lift.lift_pick(lift.OP_ASUM, 1 << 12)
    finally:
        lift.lift_set_policy(lift.POLICY_FIXED)


@pytest.mark.parametrize("env", [{"LIFT_VARIANT": "no_such_variant"}, {"LIFT_POLICY": "fastest"},
                                 {"LIFT_POLICY": "table"}, {"LIFT_POLICY": "mlp:/nonexistent"}])
def test_bad_overrides_fail_loudly(env):
    from paper_1502_02389_gb300 import lift
    assert probe(env)["rc"] == lift.ERR_INVALID_ARG
