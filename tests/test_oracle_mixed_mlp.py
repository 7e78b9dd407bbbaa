"""Pins of the mixed-precision decoders (format definitions) and of the FP64
MLP reference (finite differences, closed-form Adam step)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from oracle import mixed, mlp
from paper_1502_02389_gb300 import synth


def floats(s):
    return [float(t) for t in s.split()]


def hexes(s):
    return [int(t, 16) for t in s.split()]


def test_e4m3_goldens():
    g = read_golden("fp_formats.txt")
    vals, bits = floats(g["e4m3_values"]), hexes(g["e4m3_bits"])
    assert mixed.decode_e4m3(np.array(bits, np.uint8)).tolist() == vals
    assert synth.encode_e4m3(np.array(vals)).tolist() == bits
    ties = synth.encode_e4m3(np.array(floats(g["e4m3_ties_in"])))
    assert mixed.decode_e4m3(ties).tolist() == floats(g["e4m3_ties_out"])
    assert math.isnan(mixed.decode_e4m3(np.array([0x7F], np.uint8))[0])
    assert mixed.decode_e4m3(np.array([0x80], np.uint8))[0] == 0.0


def test_e4m3_decode_covers_every_code():
    # every finite code decodes to a value of <= 4 significant bits in the
    # E4M3 range, codes are monotone on each sign, and encode inverts decode
    codes = np.arange(256, dtype=np.uint8)
    v = mixed.decode_e4m3(codes)
    fin = ~np.isnan(v)
    assert fin.sum() == 254
    pos = v[:128][fin[:128]]
    assert np.all(np.diff(pos) > 0) and pos.max() == 448.0
    back = synth.encode_e4m3(v[fin])
    assert np.array_equal(mixed.decode_e4m3(back), v[fin])


def test_bf16_goldens():
    g = read_golden("fp_formats.txt")
    vals, bits = floats(g["bf16_values"]), hexes(g["bf16_bits"])
    assert mixed.decode_bf16(np.array(bits, np.uint16)).tolist() == vals
    assert synth.encode_bf16(np.array(vals)).tolist() == bits
    ties = synth.encode_bf16(np.array(floats(g["bf16_ties_in"])))
    assert mixed.decode_bf16(ties).tolist() == floats(g["bf16_ties_out"])


def test_bf16_rounding_error_bound():
    x = np.random.default_rng(0).standard_normal(100000) * 1e3
    r = mixed.decode_bf16(synth.encode_bf16(x))
    # RNE with 8 significant bits: relative error <= 2^-8
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))


def test_fp8_blocks_and_stored_values():
    x, _ = synth.mixed_values(10000, seed=4, two=False)
    q, s = synth.encode_fp8_blocks(x)
    assert s.size == math.ceil(10000 / 4096)
    v = mixed.stored_values("fp8", q, s)
    # each block's scale maps its amax to 448 (within fp32 rounding of s)
    for b in range(s.size):
        blk = x[b * 4096:(b + 1) * 4096]
        assert abs(np.abs(blk).max() / s[b] - 448) <= 448 * 2 ** -23
    # E4M3 relative spacing 2^-3 -> RNE error <= 2^-4 relative for normals,
    # and at most half a subnormal step (2^-10 * s) otherwise
    err = np.abs(v - x)
    bound = np.maximum(2.0 ** -4 * np.abs(x), 2.0 ** -10 * s[np.arange(x.size) // 4096])
    assert np.all(err <= bound * (1 + 1e-12))


def test_mixed_definitions_brute_force():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(9000)
    y = rng.standard_normal(9000)
    qx, sx = synth.encode_fp8_blocks(x)
    qy, sy = synth.encode_fp8_blocks(y)
    vx = mixed.stored_values("fp8", qx, sx)
    vy = mixed.stored_values("fp8", qy, sy)
    exact = sum(Fraction(a) * Fraction(b) for a, b in zip(vx[:500], vy[:500]))
    got = mixed.dot("fp8", qx[:500], sx, qy[:500], sy)
    terms = float(sum(abs(Fraction(a) * Fraction(b)) for a, b in zip(vx[:500], vy[:500])))
    assert abs(got - float(exact)) <= 500 * 2 ** -53 * terms + 1e-300
    bx = synth.encode_bf16(x[:300])
    vb = mixed.decode_bf16(bx)
    assert mixed.asum("bf16", bx) == float(sum(abs(Fraction(v)) for v in vb))


# ---------------------------------------------------------------------------
# MLP
# ---------------------------------------------------------------------------
def _params(rng, d_in=10, h=8, v=5):
    return {"W1": rng.standard_normal((d_in, h)) * 0.5, "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) * 0.5, "b2": rng.standard_normal(h) * 0.1,
            "W3": rng.standard_normal((h, v)) * 0.5, "b3": rng.standard_normal(v) * 0.1}


def test_mlp_forward_closed_form():
    # identity-like weights: with X >= 0 the ReLUs pass everything through,
    # so P = X @ W1 @ W2 @ W3 + biases propagate linearly.
    p = {"W1": np.eye(3), "b1": np.zeros(3), "W2": 2 * np.eye(3), "b2": np.ones(3),
         "W3": np.array([[1.0], [1.0], [1.0]]), "b3": np.array([0.5])}
    X = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    P, _ = mlp.forward(p, X)
    assert P.tolist() == [[2 * 6 + 3 + 0.5], [3 + 0.5]]
    # a negative pre-activation is cut by the ReLU
    P, _ = mlp.forward(p, np.array([[-1.0, 0.0, 0.0]]))
    assert P.tolist() == [[3.5]]


def test_masked_mse_by_hand():
    P = np.array([[1.0, 2.0], [3.0, 4.0]])
    T = np.array([[0.0, 2.0], [1.0, 100.0]])
    M = np.array([[1, 1], [1, 0]])
    assert mlp.masked_mse(P, T, M) == (1 + 0 + 4) / 3


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    p = _params(rng)
    X = rng.standard_normal((7, 10))
    T = rng.standard_normal((7, 5))
    M = (rng.random((7, 5)) < 0.6).astype(float)
    M[0, 0] = 1
    _, g = mlp.loss_and_grads(p, X, T, M)
    h = 1e-6
    for k in mlp.PARAM_NAMES:
        flat = p[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.masked_mse(mlp.forward(p, X)[0], T, M)
            flat[idx] = old - h
            lm = mlp.masked_mse(mlp.forward(p, X)[0], T, M)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, idx, fd, an)


def test_adam_first_step_closed_form():
    # t = 1: mhat = g, vhat = g^2, so the step is lr * g / (|g| + eps)
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    z = {"w": np.zeros(3)}
    newp, m, v = mlp.adam_step(p, g, z, z, 1, lr=0.01, eps=1e-8)
    exp = p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(newp["w"], exp, rtol=0, atol=1e-15)
    assert np.allclose(m["w"], 0.1 * g["w"]) and np.allclose(v["w"], 0.001 * g["w"] ** 2)
