"""The batched persistent launch: every op of a batch against the oracle --
bit for bit against the low-level expression its work items evaluate, and
within the tolerance of the FP64 definitions -- across graph replays, and on
the full batched workload (20,000 ops, about 60 GB) on a sample of ops."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blas
from oracle import lowlevel as ll
from oracle.patterns import C, Map, Zip, add, evaluate, mult_by
from paper_1502_02389_gb300 import synth

pytestmark = pytest.mark.gpu

VEC_MODES = [(1, 4), (4, 1), (4, 2), (4, 4), (8, 1), (8, 2)]
GEMV_VW = [1, 4, 8]


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


def expected(L, d, data, choice):
    """Expected fp32 output of one op from the oracle's expressions."""
    variant, mode, item = choice
    op = d["op"]
    if op in (L.OP_ASUM, L.OP_DOT):
        vw, j = VEC_MODES[mode]
        tile = 256 * vw * j
        name = "asum" if op == L.OP_ASUM else "dot"
        e, Lp = ll.batch_reduce(name, d["n"], item, tile, vw)
        xp = np.zeros(Lp, np.float32)
        xp[:d["n"]] = data["x"]
        if op == L.OP_ASUM:
            return evaluate(e, xp, mode="f32")
        yp = np.zeros(Lp, np.float32)
        yp[:d["n"]] = data["y"]
        return evaluate(e, (xp, yp), mode="f32")
    if op == L.OP_SCAL:
        return (data["x"].astype(np.float64) * d["alpha"]).astype(np.float32)
    M, N = d["M"], d["N"]
    vw = GEMV_VW[mode]
    z = evaluate(ll.gemv_z_variant(M, N, d["alpha"], vw, 32, 1), data["A"], mode="f32",
                 env={"x": data["x"]})
    by = evaluate(Map(mult_by(d["beta"])), data["out0"], mode="f32")
    return evaluate(C(Map(add), Zip()), (z, by), mode="f32") if d["beta"] != 0 else z


def make_small_batch(L, seed=0):
    rng = np.random.default_rng(seed)
    descs, datas, keep = [], [], []
    sizes = [0, 1, 7, 255, 256, 1000, 4097, 65536, 70001, 300000, 1 << 20]
    for i in range(150):
        kind = i % 4
        off = int(rng.integers(0, 3)) if i % 5 == 0 else 0      # some unaligned pointers
        variant = -1 if i % 3 else int(rng.integers(0, 43 if kind < 2 else (15 if kind == 2 else 8)))
        if kind == 3:
            M, N = int(rng.integers(1, 300)), int(rng.choice([1, 33, 128, 1000, 4096]))
            A = rng.standard_normal((M, N)).astype(np.float32)
            x = rng.standard_normal(N).astype(np.float32)
            y0 = rng.standard_normal(M).astype(np.float32)
            Ad, xd = torch.from_numpy(A).cuda(), torch.from_numpy(x).cuda()
            yd = torch.from_numpy(y0).cuda()
            beta = 0.5 if i % 2 else 0.0
            descs.append({"op": L.OP_GEMV, "variant": variant, "M": M, "N": N, "lda": N,
                          "alpha": 1.25, "beta": beta, "A": Ad, "x": xd, "out": yd})
            datas.append({"A": A, "x": x, "out0": y0})
            keep += [Ad, xd, yd]
            continue
        n = int(sizes[i % len(sizes)])
        x = rng.standard_normal(n).astype(np.float32)
        xb = torch.zeros(n + 8, device="cuda")
        xb[off:off + n] = torch.from_numpy(x).cuda()
        xp = xb.data_ptr() + 4 * off
        d = {"op": [L.OP_ASUM, L.OP_DOT, L.OP_SCAL][kind], "variant": variant, "n": n, "x": xp}
        data = {"x": x}
        keep.append(xb)
        if kind == 1:
            y = rng.standard_normal(n).astype(np.float32)
            yb = torch.zeros(n + 8, device="cuda")
            yb[off:off + n] = torch.from_numpy(y).cuda()
            d["y"] = yb.data_ptr() + 4 * off
            data["y"] = y
            keep.append(yb)
        if kind == 2:
            ob = torch.zeros(n + 8, device="cuda")
            d["out"] = ob.data_ptr() + 4 * off
            d["alpha"] = 1.5
            keep.append(ob)
            data["outbuf"], data["off"] = ob, off
        else:
            ob = torch.full((1,), -3.0, device="cuda")
            d["out"] = ob
            keep.append(ob)
            data["outbuf"], data["off"] = ob, 0
        descs.append(d)
        datas.append(data)
    return descs, datas, keep


def read_out(L, d, data):
    if d["op"] == L.OP_GEMV:
        return d["out"].cpu().numpy()
    if d["op"] == L.OP_SCAL:
        return data["outbuf"][data["off"]:data["off"] + d["n"]].cpu().numpy()
    return data["outbuf"].cpu().numpy()


@pytest.mark.parametrize("schedule", [0, 1])      # LIFT_BATCH_QUEUE, LIFT_BATCH_PER_ITEM
def test_small_batch_bit_exact_and_replayable(L, schedule):
    descs, datas, keep = make_small_batch(L)
    h = L.lift_batch_create(descs)
    try:
        L.lift_batch_set_schedule(h, schedule)
        info = L.lift_batch_info(h)
        assert info["items"] >= len(descs) - sum(1 for d in descs if d["op"] == L.OP_SCAL and d["n"] == 0)
        if schedule == L.BATCH_PER_ITEM:
            assert info["grid"] == info["items"]
        for rep in range(2):
            if rep:   # gemv updates y in place: restore it before the replay
                for d, data in zip(descs, datas):
                    if d["op"] == L.OP_GEMV:
                        d["out"].copy_(torch.from_numpy(data["out0"]))
            L.lift_batch_run(h)
            torch.cuda.synchronize()
            for i, (d, data) in enumerate(zip(descs, datas)):
                choice = L.lift_batch_op_choice(h, i)
                got = read_out(L, d, data)
                exp = np.asarray(expected(L, d, data, choice), np.float32).reshape(-1)
                assert np.array_equal(got.view(np.uint32) if got.size else got,
                                      exp.view(np.uint32) if exp.size else exp) or \
                    np.array_equal(got, exp), (i, d["op"], choice, got[:3], exp[:3])
                if d["op"] == L.OP_ASUM and d["n"]:
                    ref = blas.asum(data["x"].astype(np.float64))
                    assert abs(float(got[0]) - ref) <= blas.tolerance(d["n"], blas.asum_terms(data["x"]))
    finally:
        L.lift_batch_destroy(h)


def test_schedules_agree_bit_for_bit(L):
    """The two schedules of the batch (queue and one CTA per item) are the
    same expression: switching between runs of one batch re-captures its
    graph and leaves every output bit unchanged."""
    descs, datas, keep = make_small_batch(L, seed=5)
    h = L.lift_batch_create(descs)
    outs = []
    try:
        for schedule in (L.BATCH_QUEUE, L.BATCH_PER_ITEM, L.BATCH_QUEUE):
            for d, data in zip(descs, datas):
                if d["op"] == L.OP_GEMV:
                    d["out"].copy_(torch.from_numpy(data["out0"]))
            L.lift_batch_set_schedule(h, schedule)
            L.lift_batch_run(h)
            torch.cuda.synchronize()
            outs.append([read_out(L, d, data).copy() for d, data in zip(descs, datas)])
        for a, b in zip(outs[0], outs[1]):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        for a, b in zip(outs[0], outs[2]):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        with pytest.raises(L.LiftError):
            L.lift_batch_set_schedule(h, 2)
    finally:
        L.lift_batch_destroy(h)


def test_batch_uses_the_policy_pick(L):
    x = torch.randn(1 << 16, device="cuda")
    out = torch.zeros(1, device="cuda")
    L.lift_set_variant(L.OP_ASUM, 12)             # t2048_v4 -> mode (4, 2)
    try:
        h = L.lift_batch_create([{"op": L.OP_ASUM, "variant": -1, "n": 1 << 16, "x": x, "out": out}])
        v, mode, item = L.lift_batch_op_choice(h, 0)
        assert v == 12 and VEC_MODES[mode] == (4, 2) and item % 2048 == 0
        L.lift_batch_destroy(h)
    finally:
        L.lift_set_variant(L.OP_ASUM, -1)


def test_full_batched_workload_sampled(L):
    ops = synth.batch_ops()
    lay, total = synth.batch_layout(ops)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    pool = torch.randn(total, device="cuda", generator=g)
    base = pool.data_ptr()
    descs = []
    for d, e in zip(ops, lay):
        q = {"op": d["op"], "variant": -1, "n": d["n"], "M": d["M"], "N": d["N"], "lda": d["N"],
             "alpha": 1.0, "beta": 0.5, "out": base + 4 * e["out"]}
        for k in ("x", "y", "A"):
            if k in e:
                q[k] = base + 4 * e[k]
        descs.append(q)
    rng = np.random.default_rng(7)
    sample = rng.choice(len(ops), 600, replace=False)
    y0 = {int(i): pool[lay[i]["out"]:lay[i]["out"] + ops[i]["M"]].cpu().numpy()
          for i in sample if ops[i]["op"] == synth.GEMV}
    h = L.lift_batch_create(descs)
    try:
        info = L.lift_batch_info(h)
        assert 50e9 < info["bytes"] < 70e9
        L.lift_batch_run(h)
        torch.cuda.synchronize()
        for i in sample:
            i = int(i)
            d, e = ops[i], lay[i]
            get = lambda k, c: pool[e[k]:e[k] + c].cpu().numpy().astype(np.float64)  # noqa: E731
            if d["op"] == synth.GEMV:
                A = get("A", d["M"] * d["N"]).reshape(d["M"], d["N"])
                x = get("x", d["N"])
                ref = blas.gemv(A, x, y0[i].astype(np.float64), 1.0, 0.5)
                tol = blas.tolerance(d["N"], 1.0) * blas.gemv_row_terms(A, x, y0[i], 1.0, 0.5)
                got = pool[e["out"]:e["out"] + d["M"]].cpu().numpy()
                assert np.all(np.abs(got - ref) <= tol), i
            else:
                x = get("x", d["n"])
                if d["op"] == synth.ASUM:
                    ref, terms = blas.asum(x), blas.asum_terms(x)
                else:
                    y = get("y", d["n"])
                    ref, terms = blas.dot(x, y), blas.dot_terms(x, y)
                got = float(pool[e["out"]].item())
                assert abs(got - ref) <= blas.tolerance(d["n"], terms), (i, got, ref)
    finally:
        L.lift_batch_destroy(h)
