"""The C-ABI library loads and exports every entry point include/lift.h
declares; host-only calls behave as documented (no GPU needed)."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\*?\s+(lift_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_02389_gb300 import build, lift
    build.build()
    return lift.lib()


def test_every_declared_symbol_is_exported(lib):
    from paper_1502_02389_gb300 import lift
    names = header_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers every declared entry point under the same name
    assert set(names) <= set(lift.exported_symbols())


def test_status_strings(lib):
    from paper_1502_02389_gb300 import lift
    assert lift.status_string(0) == "ok"
    assert "invalid" in lift.status_string(1)
    assert lift.status_string(99) == "unknown status"


def test_variant_registry_host_side(lib):
    from paper_1502_02389_gb300 import lift
    for op in (lift.OP_ASUM, lift.OP_DOT):
        vs = lift.variants(op)
        assert len(vs) >= 30
        for v in vs:
            assert v["tile"] % (v["threads"] * v["vw"]) == 0
            assert v["tile"] in (256, 512, 1024, 2048, 4096) and v["vw"] in (1, 4, 8)
        tiles = {v["tile"] for v in vs}
        assert tiles == {256, 512, 1024, 2048, 4096}
        assert {v["passes"] for v in vs} == {1, 2}
        assert {v["tree"] for v in vs} == {0, 1, 2}
        assert {v["stride"] for v in vs} == {0, 1}
        assert any(v["stages"] > 0 for v in vs) and any(v["stages"] == 0 for v in vs)
        assert len({v["name"] for v in vs}) == len(vs)
    assert len(lift.variants(lift.OP_SCAL)) >= 10
    assert len(lift.variants(lift.OP_GEMV)) >= 5
    with pytest.raises(lift.LiftError):
        lift.lift_variant_describe(lift.OP_ASUM, 10 ** 6)


def test_features_follow_their_definition(lib):
    from paper_1502_02389_gb300 import lift
    f = lift.lift_features(lift.OP_DOT, 1 << 20)
    assert len(f) == lift.NUM_FEATURES
    assert f[:4] == [0, 1, 0, 0] and f[7:] == [1, 0, 0, 0, 0]
    assert math.isclose(f[4], math.log2(2 ** 20 + 1) / 32, rel_tol=1e-6)
    g = lift.lift_features(lift.OP_GEMV, 0, 4096, 1024)
    assert g[3] == 1 and math.isclose(g[4], math.log2(4096 * 1024 + 1) / 32, rel_tol=1e-6)
    assert math.isclose(g[5], math.log2(4097) / 16, rel_tol=1e-6)
    assert math.isclose(g[6], math.log2(1025) / 16, rel_tol=1e-6)
    assert g[10:] == [1, 1]                       # 1024 % 4 == 0 and 1024 % 8 == 0
    h = lift.lift_features(lift.OP_ASUM_FP8, 100)
    assert h[0] == 1 and h[9] == 1
    assert lift.lift_features(lift.OP_GEMV, 0, 10, 96)[10:] == [1, 1]
    assert lift.lift_features(lift.OP_GEMV, 0, 10, 97)[10:] == [0, 0]


def test_invalid_arguments_rejected_before_any_launch(lib):
    from paper_1502_02389_gb300 import lift
    # no device state: a valid call reports "not initialised"; invalid ones
    # are rejected by validation first
    with pytest.raises(lift.LiftError) as e:
        lift.lift_asum_v(0, 0, -1, 8, None, 0)
    assert e.value.status == lift.ERR_INVALID_ARG
    with pytest.raises(lift.LiftError) as e:
        lift.lift_gemv_v(0, 4, 8, 1.0, 16, 4, 32, 1.0, 48, 0)   # lda < N
    assert e.value.status == lift.ERR_INVALID_ARG
    with pytest.raises(lift.LiftError) as e:
        lift.lift_scal_v(0, 100, 1.0, 4096, 4096 + 8, 0)       # partial overlap
    assert e.value.status == lift.ERR_INVALID_ARG
    with pytest.raises(lift.LiftError) as e:
        lift.lift_asum_ex(lift.BF16, 4096, 8192, 10, 64, None, 0)  # bf16 takes no scales
    assert e.value.status == lift.ERR_INVALID_ARG
    with pytest.raises(lift.LiftError) as e:
        lift.lift_batch_set_schedule(None, lift.BATCH_PER_ITEM)   # no batch
    assert e.value.status == lift.ERR_INVALID_ARG
    assert lift.lift_batch_schedule(None) == -1


def test_batch_create_rejects_bad_descriptors_before_any_device_work(lib):
    from paper_1502_02389_gb300 import lift
    good = {"op": lift.OP_ASUM, "variant": -1, "n": 10, "x": 4096, "out": 8192}
    bad = [
        dict(good, op=lift.OP_ASUM_FP8),            # op id not supported by the batch
        dict(good, op=99),                           # op id out of range
        dict(good, variant=10 ** 5),                 # variant id out of range
        dict(good, n=-1),
        dict(good, x=0),                             # NULL x with n > 0
        dict(good, out=0),
        dict(good, x=4098),                          # not 4-byte aligned
        {"op": lift.OP_GEMV, "variant": -1, "M": 4, "N": 8, "lda": 7, "x": 64, "A": 128, "out": 256},
        {"op": lift.OP_DOT, "variant": -1, "n": 5, "x": 64, "y": 0, "out": 256},
    ]
    for d in bad:
        with pytest.raises(lift.LiftError) as e:
            lift.lift_batch_create([good, d])
        assert e.value.status == lift.ERR_INVALID_ARG, d
        assert "batch op 1" in lift.lib().lift_last_error().decode()


def test_fixed_policy_defaults_name_registered_variants(lib):
    """Each op's FIXED default (kDefaultName in csrc/api.cu, indexed by op
    id) is a variant of that op: a name that no longer matches would make the
    FIXED policy fall back silently to the op's first variant."""
    from paper_1502_02389_gb300 import lift
    src = open(os.path.join(ROOT, "paper_1502_02389_gb300", "csrc", "api.cu")).read()
    body = re.search(r"kDefaultName\[LIFT_NUM_OPS\]\s*=\s*\{(.*?)\};", src, re.S).group(1)
    names = re.findall(r'"([^"]+)"', body)
    assert len(names) == lift.NUM_OPS
    for op, name in enumerate(names):
        assert name in {v["name"] for v in lift.variants(op)}, (lift.OP_NAMES[op], name)
