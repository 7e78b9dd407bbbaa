"""The cost model's GPU kernels against the FP64 oracle (oracle/mlp.py):
forward, masked-MSE loss, gradients, Adam; and training that fits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp
from paper_1502_02389_gb300 import costmodel as cm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    return lift


def _problem(B, V, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((B, cm.D_IN)).astype(np.float32)
    T = rng.standard_normal((B, V)).astype(np.float32)
    M = (rng.random((B, V)) < 0.3).astype(np.float32)
    return X, T, M


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-30, np.max(np.abs(b))))


@pytest.mark.parametrize("B", [1, 37, 1200])
def test_forward_loss_and_gradients_match_oracle(L, B):
    _, V = cm.offsets()   # the library's current variant count
    X, T, M = _problem(B, V, B)
    tr = cm.Trainer(X, T, M, seed=3)
    loss, g = tr.grads()
    torch.cuda.synchronize()
    P = tr.P.cpu().numpy()
    params = cm.unflatten(tr.params(), V)
    Pref, cache = mlp.forward(params, X.astype(np.float64))
    assert _rel(P, Pref) <= 1e-5
    lref = mlp.masked_mse(Pref, T.astype(np.float64), M)
    assert abs(float(loss.item()) - lref) <= 1e-5 * lref
    gref = mlp.backward(params, cache, Pref, T.astype(np.float64), M)
    gg = cm.unflatten(g.cpu().numpy(), V)
    for k in mlp.PARAM_NAMES:
        assert _rel(gg[k], gref[k]) <= 1e-4, k


def test_adam_steps_match_oracle(L):
    _, V = cm.offsets()   # the library's current variant count
    X, T, M = _problem(64, V, 9)
    tr = cm.Trainer(X, T, M, seed=4)
    p = cm.unflatten(tr.params(), V)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(val) for k, val in p.items()}
    for t in (1, 2, 3):
        _, g = tr.grads()
        gh = cm.unflatten(g.cpu().numpy(), V)
        p, m, v = mlp.adam_step(p, gh, m, v, t, lr=1e-2)
        tr.t = t - 1
        tr.step(1e-2)
        got = cm.unflatten(tr.params(), V)
        for k in mlp.PARAM_NAMES:
            assert np.max(np.abs(got[k] - p[k])) <= 1e-5 * max(1.0, np.max(np.abs(p[k]))), (t, k)
        p = got   # continue from the GPU state (fp32)


def test_training_fits_a_smooth_target(L):
    _, V = cm.offsets()   # the library's current variant count
    rng = np.random.default_rng(1)
    X = rng.random((800, cm.D_IN)).astype(np.float32)
    W = rng.standard_normal((cm.D_IN, V)).astype(np.float32)
    T = np.tanh(X @ W).astype(np.float32)
    M = np.ones_like(T)
    tr = cm.Trainer(X, T, M, seed=2)
    hist = tr.train(steps=1500, lr=3e-3, log_every=100)
    assert hist[-1] < 0.05 * hist[0], hist
