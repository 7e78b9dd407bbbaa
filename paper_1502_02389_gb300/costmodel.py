"""Variant cost model: an MLP that proposes the kernel variant for a call.

The paper fixes the integer parameters of each device's expression by
exploring values empirically (Sec. 6.2) and names a model-guided search as
future work (Sec. 6.3).  Here the autotuner's measurements (``tune.py``)
train a small network that maps the features of a call (``lift_features``:
op family, log2 sizes, element type) to one predicted value per kernel
variant: the log of the variant's time relative to the fastest variant of
that shape.  The library's MLP policy picks the argmin over the op's
variants; exhaustive autotuning stays the fallback and the yardstick of
the pick's regret t(pick) / t(best).

Training runs on the GPU through the library's own kernels
(``lift_mlp_forward`` / ``_loss`` / ``_backward`` / ``_adam``); this module
only arranges the data and calls them.
"""
from __future__ import annotations

import math
import os
import time
from collections import defaultdict
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import lift, tune

D_IN, H1, H2 = lift.NUM_FEATURES, 64, 64
DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
WEIGHTS = os.path.join(DATA, "mlp_gb300.txt")   # trained on the GB300 sweep


def offsets(records: Optional[List[Dict]] = None) -> Tuple[List[int], int]:
    """Output index of each op's variant 0, and the total output width V.
    With training records, an op's slice covers the variants measured there
    (a variant added to the library later stays out of the model's picks
    until the model is retrained); otherwise the library's current lists."""
    off, v = [], 0
    for op in range(lift.MLP_OPS):
        off.append(v)
        if records is None:
            v += lift.lift_variant_count(op)
        else:
            ids = [r["variant"] for r in records if r["op"] == op]
            v += (max(ids) + 1) if ids else 0
    return off, v


def group(records: List[Dict]) -> Dict[Tuple[int, int, int, int], Dict[int, float]]:
    """(op, n, M, N) -> {variant: ms}"""
    g: Dict = defaultdict(dict)
    for r in records:
        g[(r["op"], r["n"], r["M"], r["N"])][r["variant"]] = r["ms"]
    return g


def runs_as_itself(op: int, variant: int, N: int) -> bool:
    """Whether a variant runs as itself (not its guarded fallback) on a dense
    call with aligned pointers: gemv and gemv-T rows of N floats must be a
    whole number of the variant's vectors (and of 16-byte granules for the
    bulk-copy gemv and gemv-T).  The same test the library's learned picks
    apply."""
    if op not in (lift.OP_GEMV, lift.OP_GEMV_T):
        return True
    d = lift.lift_variant_describe(op, variant)
    if (4 * N) % (4 * d["vw"]) != 0:
        return False
    if op == lift.OP_GEMV and d["tree"] == 3 and N % 256 != 0:     # tensor-copy staging
        return False
    return not (d["stages"] > 0 and (N == 0 or N % 4 != 0))


def dataset(records: List[Dict], off: Optional[List[int]] = None, V: Optional[int] = None):
    """Features X [B, D_IN], targets T [B, V] = log(t_v / t_best), mask M
    (the output slices follow ``offsets(records)`` unless given).  A timing
    of a variant that ran its fallback on that shape is masked out: the
    picks never choose such a variant there."""
    if off is None:
        off, V = offsets(records)
    g = group(records)
    keys = sorted(g)
    X = np.zeros((len(keys), D_IN), np.float32)
    T = np.zeros((len(keys), V), np.float32)
    M = np.zeros((len(keys), V), np.float32)
    for i, k in enumerate(keys):
        op, n, Mm, N = k
        X[i] = lift.lift_features(op, n, Mm, N)
        times = g[k]
        best = min(times.values())
        for v, ms in times.items():
            T[i, off[op] + v] = math.log(ms / best)
            M[i, off[op] + v] = 1.0 if runs_as_itself(op, v, N) else 0.0
    return keys, X, T, M


def init_params(V: int, seed: int = 0) -> np.ndarray:
    """He-initialised weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((D_IN, H1)) * math.sqrt(2.0 / D_IN), np.zeros(H1),
             rng.standard_normal((H1, H2)) * math.sqrt(2.0 / H1), np.zeros(H2),
             rng.standard_normal((H2, V)) * math.sqrt(1.0 / H2), np.zeros(V)]
    flat = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
    assert flat.size == lift.lift_mlp_param_count(D_IN, H1, H2, V)
    return flat


def unflatten(flat: np.ndarray, V: int) -> Dict[str, np.ndarray]:
    shapes = [("W1", (D_IN, H1)), ("b1", (H1,)), ("W2", (H1, H2)), ("b2", (H2,)),
              ("W3", (H2, V)), ("b3", (V,))]
    out, o = {}, 0
    for name, shp in shapes:
        c = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + c], np.float64).reshape(shp)
        o += c
    return out


class Trainer:
    """Full-batch Adam on the GPU with the library's MLP kernels."""

    def __init__(self, X: np.ndarray, T: np.ndarray, M: np.ndarray, seed: int = 0,
                 params: Optional[np.ndarray] = None):
        import torch
        self.torch = torch
        self.B, self.V = T.shape
        dev = "cuda"
        self.X = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
        self.T = torch.from_numpy(np.ascontiguousarray(T)).to(dev)
        self.M = torch.from_numpy(np.ascontiguousarray(M)).to(dev)
        self.inv = float(1.0 / max(1.0, M.sum()))
        p = init_params(self.V, seed) if params is None else params
        self.p = torch.from_numpy(p.copy()).to(dev)
        self.count = self.p.numel()
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.work = torch.zeros(lift.lift_mlp_work_count(self.B, H1, H2), device=dev)
        self.P = torch.zeros((self.B, self.V), device=dev)
        self.dP = torch.zeros_like(self.P)
        self.loss = torch.zeros(1, device=dev)
        self.t = 0

    def forward(self):
        lift.lift_mlp_forward(D_IN, H1, H2, self.V, self.p, self.X, self.B, self.work, self.P)
        return self.P

    def grads(self):
        """Loss and parameter gradients at the current parameters."""
        self.forward()
        lift.lift_mlp_loss(self.P, self.T, self.M, self.B * self.V, self.inv, self.dP, self.loss)
        lift.lift_mlp_backward(D_IN, H1, H2, self.V, self.p, self.X, self.B, self.work, self.dP,
                               self.g)
        return self.loss, self.g

    def step(self, lr: float):
        self.grads()
        self.t += 1
        lift.lift_mlp_adam(self.p, self.g, self.m, self.v, self.count, self.t, lr, 0.9, 0.999, 1e-8)

    def train(self, steps: int = 4000, lr: float = 3e-3, log_every: int = 0) -> List[float]:
        hist = []
        for i in range(steps):
            frac = i / max(1, steps - 1)
            self.step(lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * frac))))
            if log_every and (i % log_every == 0 or i == steps - 1):
                hist.append(float(self.loss.item()))
        self.torch.cuda.synchronize()
        return hist

    def params(self) -> np.ndarray:
        return self.p.cpu().numpy()


def box(records: List[Dict]) -> Dict[int, Tuple[float, ...]]:
    """Per op, the trained range in log2(size + 1): (lo, hi) of n (M*N for
    gemv and gemv-T), of M and of N -- what LIFT_POLICY_MLP_TUNE treats as
    inside the model's experience."""
    out = {}
    for op in sorted({r["op"] for r in records}):
        rs = [r for r in records if r["op"] == op]
        mat = op in (lift.OP_GEMV, lift.OP_GEMV_T)
        cols = [[math.log2((r["M"] * r["N"] if mat else r["n"]) + 1) for r in rs],
                [math.log2(r["M"] + 1) for r in rs], [math.log2(r["N"] + 1) for r in rs]]
        out[op] = tuple(v for c in cols for v in (min(c), max(c)))
    return out


def save(path: str, params: np.ndarray, V: int, off: Optional[List[int]] = None,
         records: Optional[List[Dict]] = None) -> None:
    """Weights file read by lift_set_policy(LIFT_POLICY_MLP[_TUNE], path);
    ``off`` are the output slices of the training data
    (``offsets(records)``); with the training records, the trained range of
    each op is appended ("box")."""
    if off is None:
        off, _ = offsets()
    with open(path, "w") as f:
        f.write(f"lift-mlp 2 {D_IN} {H1} {H2} {V}\n")
        f.write(f"offsets {len(off)} " + " ".join(str(o) for o in off) + "\n")
        f.write(" ".join(f"{x:.9g}" for x in params.tolist()) + "\n")
        if records:
            b = box(records)
            f.write(f"box {len(b)}\n")
            for op, v in b.items():
                f.write(f"{op} " + " ".join(f"{x:.6f}" for x in v) + "\n")


# ---------------------------------------------------------------------------
# regret
# ---------------------------------------------------------------------------
def regrets(records: List[Dict], pick) -> np.ndarray:
    """t(pick(shape)) / t(best) over the shapes of an exhaustive sweep."""
    out = []
    for (op, n, M, N), times in sorted(group(records).items()):
        v = pick(op, n, M, N)
        out.append(times[v] / min(times.values()))
    return np.asarray(out)


def summary(r: np.ndarray) -> Dict[str, float]:
    return {"geomean": float(np.exp(np.mean(np.log(r)))), "p90": float(np.percentile(r, 90)),
            "max": float(r.max()), "shapes": int(r.size)}


def best_fixed(records: List[Dict]) -> Dict[int, int]:
    """Per op, the single variant with the smallest geomean time ratio over
    the given shapes (the paper's one fixed derivation per device)."""
    g = group(records)
    best = {}
    for op in range(lift.MLP_OPS):
        rows = [t for (o, *_), t in g.items() if o == op]
        if not rows:
            continue
        cnt = lift.lift_variant_count(op)
        score = []
        for v in range(cnt):
            if all(v in t for t in rows):
                score.append((np.mean([math.log(t[v] / min(t.values())) for t in rows]), v))
        best[op] = min(score)[1]
    return best


def evaluate_policies(train: List[Dict], heldout: List[Dict], weights: str, table: str):
    """Regret on the held-out sweep of the learned pick (MLP policy through
    lift_pick) and of the two methods without the model: the single best
    fixed variant per op and the nearest-shape tuned table."""
    res = {}
    lift.lift_set_policy(lift.POLICY_MLP, weights)
    try:
        res["mlp"] = summary(regrets(heldout, lambda op, n, M, N: lift.lift_pick(op, n, M, N)))
    finally:
        lift.lift_set_policy(lift.POLICY_FIXED)
    bf = best_fixed(train)
    res["best_fixed"] = summary(regrets(heldout, lambda op, n, M, N: bf[op]))
    tune.write_table(train, table)
    lift.lift_set_policy(lift.POLICY_TABLE, table)
    try:
        res["table"] = summary(regrets(heldout, lambda op, n, M, N: lift.lift_pick(op, n, M, N)))
    finally:
        lift.lift_set_policy(lift.POLICY_FIXED)
    return res


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the variant cost model on the GPU")
    ap.add_argument("--train", nargs="+", default=[os.path.join(DATA, "timings_gb300_train.csv")])
    ap.add_argument("--heldout", nargs="+",
                    default=[os.path.join(DATA, "timings_gb300_heldout.csv")])
    ap.add_argument("--out", required=True)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workloads", default=None,
                    help="timings of the benchmark shapes, added to the training set with weight")
    ap.add_argument("--workload-weight", type=int, default=20,
                    help="rows each benchmark shape counts as in the loss")
    a = ap.parse_args()
    lift.lift_init()
    tr = [r for f in a.train for r in tune.load_csv(f)]
    ho = [r for f in a.heldout for r in tune.load_csv(f)]
    wl = tune.load_csv(a.workloads) if a.workloads else []
    off, V = offsets(tr + wl)
    _, X, T, M = dataset(tr, off, V)
    if wl:      # the shapes the library is benchmarked on weigh more in the loss
        _, Xw, Tw, Mw = dataset(wl, off, V)
        w = a.workload_weight
        X, T, M = (np.concatenate([A, np.repeat(B, w, axis=0)]) for A, B in ((X, Xw), (T, Tw), (M, Mw)))
    trainer = Trainer(X, T, M, seed=a.seed)
    t0 = time.perf_counter()
    hist = trainer.train(a.steps, a.lr, log_every=max(1, a.steps // 10))
    train_s = time.perf_counter() - t0      # train() ends with a device synchronise
    save(a.out, trainer.params(), V, off, tr + wl)
    res = evaluate_policies(tr + wl, ho, a.out, a.out + ".table")
    if wl:
        res["workloads"] = summary(regrets(wl, lambda op, n, M, N: _mlp_pick(a.out, op, n, M, N)))
    res.update({"loss": hist, "train_timings": len(tr), "workload_timings": len(wl),
                "heldout_timings": len(ho), "train_rows": int(X.shape[0]),
                "train_seconds": round(train_s, 3), "adam_steps": a.steps})
    print(json.dumps(res))


def _mlp_pick(weights: str, op, n, M, N) -> int:
    lift.lift_set_policy(lift.POLICY_MLP, weights)
    try:
        return lift.lift_pick(op, n, M, N)
    finally:
        lift.lift_set_policy(lift.POLICY_FIXED)


if __name__ == "__main__":
    main()
