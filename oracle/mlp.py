"""FP64 reference of the variant cost model: a multilayer perceptron with two
hidden ReLU layers, a masked mean-squared-error loss and the Adam update.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The paper leaves the choice of split sizes and vector widths to empirical
exploration (Sec. 6.2) and names search guided by performance models or
machine learning as the way to automate it (Sec. 6.3).  The model here maps
the features of a call (op, log2 sizes, dtype) to one predicted log-time per
kernel variant.

Conventions (shared by the GPU kernels only through this documentation):
  X [B, d_in];  layer k: H_k = relu(H_{k-1} @ W_k + b_k), W_k [d_{k-1}, d_k];
  output P = H_2 @ W_3 + b_3 (no activation);
  loss L = sum(M * (P - T)^2) / sum(M)   (M a 0/1 mask of measured pairs);
  Adam (Kingma and Ba, 2015):  m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
  p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(params: Dict[str, np.ndarray], X: np.ndarray):
    X = np.asarray(X, np.float64)
    Z1 = X @ params["W1"] + params["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ params["W2"] + params["b2"]
    H2 = np.maximum(Z2, 0.0)
    P = H2 @ params["W3"] + params["b3"]
    return P, (X, Z1, H1, Z2, H2)


def masked_mse(P, T, M) -> float:
    M = np.asarray(M, np.float64)
    return float(np.sum(M * (P - T) ** 2) / np.sum(M))


def backward(params, cache, P, T, M) -> Dict[str, np.ndarray]:
    X, Z1, H1, Z2, H2 = cache
    M = np.asarray(M, np.float64)
    dP = 2.0 * M * (P - T) / np.sum(M)
    g = {}
    g["W3"] = H2.T @ dP
    g["b3"] = dP.sum(axis=0)
    dH2 = dP @ params["W3"].T
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ params["W2"].T
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return g


def loss_and_grads(params, X, T, M) -> Tuple[float, Dict[str, np.ndarray]]:
    P, cache = forward(params, X)
    return masked_mse(P, T, M), backward(params, cache, P, T, M)


def adam_step(params, grads, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new params, m, v."""
    newp, newm, newv = {}, {}, {}
    for k in params:
        newm[k] = b1 * m[k] + (1 - b1) * grads[k]
        newv[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mhat = newm[k] / (1 - b1 ** t)
        vhat = newv[k] / (1 - b2 ** t)
        newp[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return newp, newm, newv
