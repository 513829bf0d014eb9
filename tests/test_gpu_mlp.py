"""The surrogate network's GPU kernels (bf16 tensor-core GEMMs, fp32
accumulation) against the FP64 oracle network: forward values, every
gradient, one Adam step, and that training fits a regression."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


def _problem(D=37, n=300, seed=0):
    g = np.random.default_rng(seed)
    p = omlp.init_params(D, 256, 256, seed=seed)
    p["b1"] = g.normal(0, 0.05, 256)
    p["b2"] = g.normal(0, 0.05, 256)
    p["b3"] = 0.1
    X = g.uniform(-1, 1, (n, D))
    t = g.normal(0, 1, n)
    return p, X, t


def _bf16_params(p):
    q = dict(p)
    for k in ("W1", "W2", "w3"):
        q[k] = omlp.bf16_round(p[k])
    for k in ("b1", "b2"):
        q[k] = np.asarray(p[k], np.float32).astype(np.float64)
    q["b3"] = float(np.float32(p["b3"]))
    return q


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30)


@pytest.mark.parametrize("D,n", [(37, 300), (200, 1024)])
def test_forward_and_gradients_match_oracle(apo, D, n):
    import torch
    p, X, t = _problem(D, n)
    net = apo.Mlp(D, seed=1)
    net.set_params(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], p["b3"])
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dt = torch.tensor(t, dtype=torch.float32, device="cuda")
    dy = torch.empty(n, device="cuda")
    net.forward(dX, dy)
    g_gpu, loss_gpu = net.gradients(dX, dt)
    q = _bf16_params(p)
    Xb = omlp.bf16_round(X)
    t32 = np.asarray(t, np.float32).astype(np.float64)
    # oracle with the GPU's storage precision (bf16 activations): tight
    y_e, c_e = omlp.forward(q, Xb, act_round=omlp.bf16_round)
    np.testing.assert_allclose(dy.cpu().numpy(), y_e, rtol=2e-3, atol=2e-3)
    g_e = omlp.backward(q, c_e, y_e, t32)
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        assert _rel(g_gpu[k], g_e[k]) < 1e-2, k
    assert loss_gpu == pytest.approx(omlp.mse(y_e, t32), rel=1e-3)
    # pure FP64 oracle on the bf16-rounded inputs and weights: within bf16 error
    y_o, c_o = omlp.forward(q, Xb)
    g_o = omlp.backward(q, c_o, y_o, t32)
    for k in ("W1", "W2", "w3"):
        assert _rel(g_gpu[k], g_o[k]) < 3e-2, k


def test_one_adam_step_matches_oracle(apo):
    import torch
    D, n = 24, 128
    p, X, t = _problem(D, n, seed=2)
    net = apo.Mlp(D, seed=2)
    net.set_params(p["W1"], p["b1"], p["W2"], p["b2"], p["w3"], p["b3"])
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dt = torch.tensor(t, dtype=torch.float32, device="cuda")
    net.train(dX, dt, steps=1, batch=n, lr=1e-3)
    torch.cuda.synchronize()
    got = net.get_params()
    q = _bf16_params(p)
    y, c = omlp.forward(q, omlp.bf16_round(X), act_round=omlp.bf16_round)
    g = omlp.backward(q, c, y, np.asarray(t, np.float32).astype(np.float64))
    m = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in p.items()}
    v = {k: np.zeros_like(np.asarray(vv, np.float64)) for k, vv in p.items()}
    master = {k: (np.asarray(p[k], np.float32).astype(np.float64) if k != "b3" else float(np.float32(p["b3"]))) for k in p}
    want = omlp.adam_step(master, g, m, v, 1, lr=1e-3)
    for k in ("W1", "b1", "W2", "b2", "w3"):
        step_gpu = np.asarray(got[k], np.float64) - master[k]
        step_orc = want[k] - master[k]
        # the first step moves every weight by about lr sign(g): compare the moves
        big = np.abs(g[k]) > 1e-4 * np.max(np.abs(g[k]))
        assert np.mean(np.sign(step_gpu[big]) == np.sign(step_orc[big])) > 0.99, k
        np.testing.assert_allclose(step_gpu[big], step_orc[big], atol=2e-5, rtol=0)


def test_training_fits_a_regression(apo):
    import torch
    g = np.random.default_rng(5)
    D, n = 16, 4096
    X = g.uniform(-1, 1, (n, D))
    t = np.sin(2 * X[:, 0]) + (X[:, 1:4] ** 2).sum(1) - 1.0
    net = apo.Mlp(D, seed=5)
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dt = torch.tensor(t, dtype=torch.float32, device="cuda")
    dy = torch.empty(n, device="cuda")
    net.forward(dX, dy)
    l0 = float(((dy.cpu().numpy() - t) ** 2).mean())
    net.train(dX, dt, steps=400, batch=512, lr=2e-3, seed=1)
    net.forward(dX, dy)
    l1 = float(((dy.cpu().numpy() - t) ** 2).mean())
    assert l1 < 0.05 * l0, (l0, l1)
