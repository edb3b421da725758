"""CPU oracle of the subtree-size MLP -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module.  It restates, in float64 numpy, what
the learned scheduler's CUDA kernels compute, so their outputs and gradients
can be checked element by element:

    h1 = relu(W1 x + b1)        W1: 64 x 8
    h2 = relu(W2 h1 + b2)       W2: 64 x 64
    y  = w3 . h2 + b3           w3: 64,  b3: scalar
    loss = mean_i (y_i - t_i)^2

The parameters the kernels use are BF16 values (rounded to nearest-even from
FP32 master copies); this oracle takes the same BF16-rounded values, widened
exactly to float64, so the only difference left is the kernels' FP32
accumulation order.  The optimiser is Adam (Kingma & Ba 2015) on the FP32
master weights; the oracle applies the published update rule in float64.

The network is not part of the paper: it orders and splits work and never
touches the integer counts (its predictions only change which warp runs which
root, never what is counted).
"""
from __future__ import annotations

import numpy as np

D_IN, D_H = 8, 64
SHAPES = {"W1": (D_H, D_IN), "b1": (D_H,), "W2": (D_H, D_H), "b2": (D_H,), "w3": (D_H,), "b3": (1,)}
ORDER = ("W1", "b1", "W2", "b2", "w3", "b3")


def bf16_round(x) -> np.ndarray:
    """FP32 -> BF16 with round-to-nearest-even, returned as float32 values
    (NaN kept quiet).  Definition: keep the top 16 bits of the IEEE-754
    binary32 word after adding 0x7FFF plus the lowest kept bit."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    r = np.where(nan, (u | 0x00400000) & 0xFFFF0000, r)
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def init_params(seed: int) -> dict[str, np.ndarray]:
    """He-uniform initialisation in FP32 (master weights)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name in ORDER:
        shape = SHAPES[name]
        if name.startswith("b"):
            p[name] = np.zeros(shape, dtype=np.float32)
        else:
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            lim = np.sqrt(6.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shape).astype(np.float32)
    return p


def flatten(p: dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float32).ravel() for k in ORDER])


def unflatten(v: np.ndarray) -> dict[str, np.ndarray]:
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(v[o:o + n]).reshape(SHAPES[k])
        o += n
    return out


N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())   # 4,801


def forward(p: dict[str, np.ndarray], X: np.ndarray):
    """Forward pass in float64 on the given parameter values; returns (y, cache)."""
    P = {k: np.asarray(v, dtype=np.float64) for k, v in p.items()}
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (X, z1, h1, z2, h2, P)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def backward(cache, t: np.ndarray) -> dict[str, np.ndarray]:
    """Gradients of the mean squared error w.r.t. every parameter (float64)."""
    X, z1, h1, z2, h2, P = cache
    B = X.shape[0]
    y = h2 @ P["w3"] + P["b3"][0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B       # dL/dy
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, P["w3"])
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(master: dict, grads: dict, m: dict, v: dict, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (bias-corrected) in float64; returns new (master, m, v)."""
    nm, nmm, nv = {}, {}, {}
    for k in ORDER:
        g = np.asarray(grads[k], dtype=np.float64)
        mk = beta1 * np.asarray(m[k], dtype=np.float64) + (1 - beta1) * g
        vk = beta2 * np.asarray(v[k], dtype=np.float64) + (1 - beta2) * g * g
        mh = mk / (1 - beta1 ** step)
        vh = vk / (1 - beta2 ** step)
        nm[k] = np.asarray(master[k], dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps)
        nmm[k], nv[k] = mk, vk
    return nm, nmm, nv


def spearman(a, b) -> float:
    """Spearman rank correlation (average ranks for ties)."""
    def ranks(x):
        x = np.asarray(x, dtype=np.float64)
        order = np.argsort(x, kind="mergesort")
        r = np.empty_like(x)
        r[order] = np.arange(x.shape[0], dtype=np.float64)
        # average ties
        xs = x[order]
        i = 0
        while i < xs.shape[0]:
            j = i
            while j + 1 < xs.shape[0] and xs[j + 1] == xs[i]:
                j += 1
            if j > i:
                r[order[i:j + 1]] = (i + j) / 2.0
            i = j + 1
        return r
    ra, rb = ranks(a), ranks(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0
