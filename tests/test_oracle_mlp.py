"""Pins the FP64 surrogate-network oracle: backward against central finite
differences, the first Adam step against its closed form, bfloat16 rounding
against torch's conversion, and a toy regression that the update rule fits."""
import numpy as np
import pytest

from oracle import mlp


def _setup(seed=0, B=16, D=12, H=24):
    g = np.random.default_rng(seed)
    p = mlp.init_params(D, H, H, seed=seed)
    p["b1"] = g.normal(0, 0.1, H)
    p["b2"] = g.normal(0, 0.1, H)
    p["b3"] = 0.3
    X = g.normal(0, 1, (B, D))
    t = g.normal(0, 1, B)
    return p, X, t


def test_backward_matches_finite_differences():
    p, X, t = _setup()
    y, cache = mlp.forward(p, X)
    # keep away from ReLU kinks so that the loss is smooth around the point
    assert np.min(np.abs(cache["Z1"])) > 1e-3 and np.min(np.abs(cache["Z2"])) > 1e-3
    g = mlp.backward(p, cache, y, t)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in ["W1", "b1", "W2", "b2", "w3", "b3"]:
        val = np.asarray(p[k], np.float64)
        idxs = [()] if val.ndim == 0 else [tuple(rng.integers(0, s) for s in val.shape) for _ in range(6)]
        for ix in idxs:
            q = {kk: np.array(vv, dtype=np.float64, copy=True) for kk, vv in p.items()}
            q[k][ix] += h
            lp = mlp.mse(mlp.forward(q, X)[0], t)
            q[k][ix] -= 2 * h
            lm = mlp.mse(mlp.forward(q, X)[0], t)
            num = (lp - lm) / (2 * h)
            ana = np.asarray(g[k])[ix]
            assert ana == pytest.approx(num, rel=1e-5, abs=1e-8), (k, ix)


def test_first_adam_step_closed_form():
    p, X, t = _setup(2)
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, t)
    m = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in p.items()}
    v = {k: np.zeros_like(np.asarray(vv, np.float64)) for k, vv in p.items()}
    q = mlp.adam_step(p, g, m, v, 1, lr=1e-3)
    # m_hat = g, v_hat = g^2: the first step moves each weight by lr g / (|g| + eps)
    for k in p:
        gk = np.asarray(g[k], np.float64)
        np.testing.assert_allclose(np.asarray(q[k]) - np.asarray(p[k]), -1e-3 * gk / (np.abs(gk) + 1e-8),
                                   rtol=1e-12, atol=1e-15)


def test_bf16_round_matches_torch():
    import torch
    a = np.random.default_rng(3).normal(0, 10, 10000).astype(np.float32)
    want = torch.tensor(a).to(torch.bfloat16).float().numpy().astype(np.float64)
    np.testing.assert_array_equal(mlp.bf16_round(a), want)


def test_training_fits_a_toy_regression():
    g = np.random.default_rng(4)
    X = g.uniform(-1, 1, (256, 4))
    t = (X ** 2).sum(1) - 1.0
    p = mlp.init_params(4, 32, 32, seed=4)
    m = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in p.items()}
    v = {k: np.zeros_like(np.asarray(vv, np.float64)) for k, vv in p.items()}
    l0 = mlp.mse(mlp.forward(p, X)[0], t)
    for step in range(1, 401):
        y, c = mlp.forward(p, X)
        p = mlp.adam_step(p, mlp.backward(p, c, y, t), m, v, step, lr=1e-2)
    assert mlp.mse(mlp.forward(p, X)[0], t) < 0.05 * l0
