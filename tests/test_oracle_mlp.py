"""Pins of the MLP oracle against things other than itself: finite
differences (analytic gradient vs numerical derivative of the loss), torch's
autograd, torch's BF16 conversion, torch's Adam, and scipy's Spearman."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as M


def _setup(seed=0, B=37):
    rng = np.random.default_rng(seed)
    p = {k: M.bf16_round(v) for k, v in M.init_params(seed).items()}
    p["b1"] = M.bf16_round(rng.normal(0, 0.1, 64))
    p["b2"] = M.bf16_round(rng.normal(0, 0.1, 64))
    p["b3"] = M.bf16_round(np.array([0.3]))
    X = rng.normal(0, 1, (B, 8)).astype(np.float32)
    t = rng.normal(0, 2, B)
    return p, X, t


def test_param_count():
    assert M.N_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-30, 100), rng.normal(0, 1e30, 100),
                        [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, np.inf, -np.inf]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = M.bf16_round(x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_gradients_finite_differences():
    p, X, t = _setup(1)
    y, cache = M.forward(p, X)
    g = M.backward(cache, t)
    rng = np.random.default_rng(9)
    P64 = {k: np.asarray(v, dtype=np.float64) for k, v in p.items()}
    for name in M.ORDER:
        flat = P64[name].ravel()
        for idx in rng.choice(flat.shape[0], size=min(6, flat.shape[0]), replace=False):
            h = 1e-6
            plus = {k: v.copy() for k, v in P64.items()}
            minus = {k: v.copy() for k, v in P64.items()}
            plus[name].ravel()[idx] += h
            minus[name].ravel()[idx] -= h
            num = (M.loss(M.forward(plus, X)[0], t) - M.loss(M.forward(minus, X)[0], t)) / (2 * h)
            ana = g[name].ravel()[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (name, idx, num, ana)


def test_forward_backward_match_torch_autograd():
    torch = pytest.importorskip("torch")
    p, X, t = _setup(2, B=64)
    y, cache = M.forward(p, X)
    g = M.backward(cache, t)
    T = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=True) for k, v in p.items()}
    Xt = torch.tensor(X.astype(np.float64))
    h1 = torch.relu(Xt @ T["W1"].T + T["b1"])
    h2 = torch.relu(h1 @ T["W2"].T + T["b2"])
    yt = h2 @ T["w3"] + T["b3"][0]
    lt = ((yt - torch.tensor(t)) ** 2).mean()
    lt.backward()
    assert np.allclose(yt.detach().numpy(), y, rtol=1e-12, atol=1e-12)
    for k in M.ORDER:
        assert np.allclose(T[k].grad.numpy(), g[k], rtol=1e-10, atol=1e-12), k


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    p, X, t = _setup(4)
    master = {k: np.asarray(v, dtype=np.float64) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in master.items()}
    v = {k: np.zeros_like(vv) for k, vv in master.items()}
    T = {k: torch.tensor(vv.copy(), requires_grad=True) for k, vv in master.items()}
    opt = torch.optim.Adam([T[k] for k in M.ORDER], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 4):
        _, cache = M.forward(master, X)
        g = M.backward(cache, t)
        master, m, v = M.adam_step(master, g, m, v, step, 1e-2)
        opt.zero_grad()
        Xt = torch.tensor(X.astype(np.float64))
        h1 = torch.relu(Xt @ T["W1"].T + T["b1"])
        h2 = torch.relu(h1 @ T["W2"].T + T["b2"])
        yt = h2 @ T["w3"] + T["b3"][0]
        ((yt - torch.tensor(t)) ** 2).mean().backward()
        opt.step()
        for k in M.ORDER:
            assert np.allclose(T[k].detach().numpy(), master[k], rtol=1e-9, atol=1e-12), (step, k)


def test_spearman_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(5)
    a = rng.integers(0, 20, 300)
    b = a + rng.integers(0, 10, 300)
    assert abs(M.spearman(a, b) - stats.spearmanr(a, b).statistic) < 1e-12
