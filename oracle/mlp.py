"""FP64 reference of the surrogate network (TEST INFRASTRUCTURE).

The surrogate that pre-screens APO candidates is a multilayer perceptron
D -> 256 -> 256 -> 1 with ReLU activations, trained on mean squared error with
Adam.  This module is the plain float64 statement of its forward pass, its
gradients and the Adam update, written from the definitions (chain rule), with
numpy matrix products as the only library step.  Only the tests and the
benchmark's CPU leg use it; the GPU kernels share none of it.

Parameters: W1 [D, H1], b1 [H1], W2 [H1, H2], b2 [H2], w3 [H2], b3 scalar.
"""
from __future__ import annotations

import numpy as np


def init_params(D, H1=256, H2=256, seed=0):
    """He-uniform initialisation (a deterministic, seeded starting point)."""
    g = np.random.default_rng(seed)
    lim1, lim2, lim3 = np.sqrt(6.0 / D), np.sqrt(6.0 / H1), np.sqrt(6.0 / H2)
    return {"W1": g.uniform(-lim1, lim1, (D, H1)), "b1": np.zeros(H1),
            "W2": g.uniform(-lim2, lim2, (H1, H2)), "b2": np.zeros(H2),
            "w3": g.uniform(-lim3, lim3, H2), "b3": 0.0}


def _ident(a):
    return a


def forward(p, X, act_round=None):
    """y = relu(relu(X W1 + b1) W2 + b2) w3 + b3; returns (y, cache).

    act_round (optional) is applied to the hidden activations H1, H2 where a
    network stores them in a narrower format (e.g. bf16_round)."""
    r = act_round or _ident
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"] + p["b1"]
    H1 = r(np.maximum(Z1, 0.0))
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = r(np.maximum(Z2, 0.0))
    y = H2 @ p["w3"] + p["b3"]
    return y, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2, "round": r}


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def backward(p, cache, y, t):
    """Gradients of L = mean((y - t)^2) with respect to every parameter (the
    hidden-layer error signals are rounded like the activations when the
    forward pass was given act_round)."""
    r = cache.get("round", _ident)
    B = y.shape[0]
    dy = 2.0 * (y - t) / B
    g = {}
    g["w3"] = cache["H2"].T @ dy
    g["b3"] = float(dy.sum())
    dZ2 = np.outer(dy, p["w3"]) * (cache["Z2"] > 0)
    g["W2"] = cache["H1"].T @ r(dZ2)
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (r(dZ2) @ p["W2"].T) * (cache["Z1"] > 0)
    g["W1"] = cache["X"].T @ r(dZ1)
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; step >= 1."""
    out = {}
    for k in p:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * np.square(g[k])
        mh = m[k] / (1.0 - beta1 ** step)
        vh = v[k] / (1.0 - beta2 ** step)
        out[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return out


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even) and back."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
