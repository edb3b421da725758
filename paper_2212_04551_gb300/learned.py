"""Learned scheduler: train the subtree-size MLP and schedule roots with it.

Orchestration only -- every arithmetic step runs in libgpm's kernels
(gpm_root_features, gpm_mlp_grad, gpm_mlp_adam, gpm_mlp_forward,
gpm_sched_from_scores, gpm_count_*); torch provides device memory.

* Training set: R-MAT graphs (scale 12, edge factor 8, seeds 100-131 by
  default); features from gpm_root_features, labels = log1p of each root's
  number of enumerated subgraphs as measured by the plain enumerator
  (gpm_count_roots with per-root output).
* Training: MSE on the log-sizes, Adam, fixed minibatches of a dataset
  shuffled once (seeded), BF16 weights refreshed from FP32 masters each step.
* Scheduling: predicted log-size per vertex -> roots ordered by prediction
  (LPT), and the roots whose predicted size exceeds a warp's fair share of
  the predicted total are pre-split into several units.
"""
from __future__ import annotations

import base64
import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import gpm
from . import graphs as G

# Trained weights shipped with the package (written by ``python -m
# paper_2212_04551_gb300.learned``): FP32 masters plus the record of the run.
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "motif_rmat12_k56.json")

D_IN, D_H = 8, 64
SHAPES = [("W1", (D_H, D_IN)), ("b1", (D_H,)), ("W2", (D_H, D_H)), ("b2", (D_H,)), ("w3", (D_H,)), ("b3", (1,))]


def init_master(seed: int) -> np.ndarray:
    """He-uniform FP32 initial weights, flat in the library's parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in SHAPES:
        if name.startswith("b"):
            parts.append(np.zeros(shape, dtype=np.float32).ravel())
        else:
            fan_in = shape[1] if len(shape) == 2 else shape[0]
            lim = math.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, size=shape).astype(np.float32).ravel())
    v = np.concatenate(parts)
    assert v.shape[0] == gpm.GPM_MLP_PARAMS
    return v


@dataclass
class Model:
    master: object            # FP32 master weights (CUDA tensor)
    w: object                 # BF16 copy as uint16 bits (CUDA tensor)
    m: object
    v: object
    step: int = 0
    history: list = field(default_factory=list)


def new_model(seed: int = 0, stream=None) -> Model:
    import torch
    master = torch.from_numpy(init_master(seed)).cuda()
    w = torch.zeros(gpm.GPM_MLP_PARAMS, dtype=torch.int16, device="cuda")
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    zero = torch.zeros_like(master)
    # an Adam step with zero gradient and zero learning rate leaves the
    # masters as they are and writes their BF16 copy
    gpm.gpm_mlp_adam(master, m, v, zero, 1, 0.0, w, stream)
    return Model(master, w, m, v)


def features(dg, n: int, k: int):
    import torch
    x = torch.empty((max(n, 1), D_IN), dtype=torch.float32, device="cuda")
    gpm.gpm_root_features(dg, k, x)
    return x[:n]


def root_sizes(dg, app: int, k: int) -> np.ndarray:
    """Per-root number of enumerated k-subgraphs (plain enumerator)."""
    _, pr = gpm.gpm_count_roots(dg, app, k, None, per_root=True)
    return pr.astype(np.float64)


def training_set(app: int = gpm.GPM_APP_MOTIF, k=5, seeds=range(100, 132), scale: int = 12,
                 edge_factor: int = 8, stream=None):
    """(X, T) on the device: features and log1p(size) of every root of every
    graph, for each size in ``k`` (an int or a sequence of ints; the size is
    feature f7, so one network learns all of them)."""
    import torch
    ks = [k] if isinstance(k, int) else list(k)
    xs, ts = [], []
    for seed in seeds:
        g = G.rmat(scale, edge_factor, 0.57, 0.19, 0.19, seed)
        dg = gpm.graph_from_csr(g, stream=stream)
        for kk in ks:
            xs.append(features(dg, g.n, kk))
            ts.append(torch.from_numpy(np.log1p(root_sizes(dg, app, kk)).astype(np.float32)).cuda())
        dg.close()
    return torch.cat(xs), torch.cat(ts)


def train(model: Model, X, T, epochs: int = 60, batch: int = 4096, lr: float = 3e-3, seed: int = 0,
          stream=None) -> Model:
    import torch
    n = int(X.shape[0])
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).cuda()
    Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
    grad = torch.zeros(gpm.GPM_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    nb = max(1, n // batch)
    for ep in range(epochs):
        ep_loss = 0.0
        for b in range(nb):
            lo, hi = b * batch, (n if b == nb - 1 else (b + 1) * batch)
            gpm.gpm_mlp_grad(model.w, Xs[lo:hi], Ts[lo:hi], grad, loss, stream)
            model.step += 1
            gpm.gpm_mlp_adam(model.master, model.m, model.v, grad, model.step, lr, model.w, stream)
            ep_loss += float(loss.item()) * (hi - lo)
        model.history.append(ep_loss / n)
    return model


def mse(model: Model, X, T, stream=None) -> float:
    import torch
    grad = torch.zeros(gpm.GPM_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gpm.gpm_mlp_grad(model.w, X, T, grad, loss, stream)
    return float(loss.item())


def predict(model: Model, X, stream=None):
    import torch
    y = torch.empty(int(X.shape[0]), dtype=torch.float32, device="cuda")
    gpm.gpm_mlp_forward(model.w, X, y, stream)
    return y


def split_plan(pred_log: np.ndarray, warps: int, chunks: int = 8, max_units: int = 1024) -> int:
    """How many of the heaviest predicted roots to pre-split: those whose
    predicted size exceeds the fair share of one warp (total / warps), up to
    max_units // chunks roots."""
    size = np.expm1(np.clip(np.asarray(pred_log, dtype=np.float64), 0, 80))
    share = size.sum() / max(warps, 1)
    heavy = int((size > share).sum())
    return min(heavy, max_units // max(chunks, 1))


def schedule(dg, app: int, pred_vertex, roots=None, warps: int = 4864, chunks: int = 8,
             balanced: bool = True, units_per_warp: int = 4, max_chunks: int = 64) -> dict:
    """Order ``roots`` (None: all) by predicted size and pre-split the
    heaviest: in proportion to the predicted size (``balanced``: about
    ``units_per_warp`` units per warp in all, at most ``max_chunks`` per
    root), or the top few into ``chunks`` units each."""
    if balanced:
        gpm.gpm_sched_balanced(dg, app, pred_vertex.contiguous(), roots, units_per_warp * warps, max_chunks)
        return {"plan": "balanced", "target_units": units_per_warp * warps, "max_chunks": max_chunks}
    pv = pred_vertex.detach().float().cpu().numpy()
    sel = pv if roots is None else pv[np.asarray(roots)]
    n_split = split_plan(sel, warps, chunks)
    gpm.gpm_sched_from_scores(dg, app, pred_vertex.contiguous(), roots, n_split, chunks if n_split else 0)
    return {"plan": "top", "split_roots": n_split, "chunks": chunks if n_split else 0}

def save(model: Model, path: str, record: dict) -> None:
    """FP32 master weights (little-endian, base64) and the training record."""
    master = model.master.detach().float().cpu().numpy().astype("<f4")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"params": gpm.GPM_MLP_PARAMS, "master_f32_b64": base64.b64encode(master.tobytes()).decode(),
                   "record": record}, f, indent=1)


def load(path: str = WEIGHTS, stream=None):
    """(Model, training record) from a file written by ``save``."""
    import torch
    with open(path) as f:
        d = json.load(f)
    master = np.frombuffer(base64.b64decode(d["master_f32_b64"]), dtype="<f4").astype(np.float32)
    if master.shape[0] != gpm.GPM_MLP_PARAMS:
        raise ValueError("weight file does not match the network")
    model = new_model(0, stream)
    model.master.copy_(torch.from_numpy(master.copy()))
    zero = torch.zeros_like(model.master)
    gpm.gpm_mlp_adam(model.master, torch.zeros_like(zero), torch.zeros_like(zero), zero, 1, 0.0, model.w, stream)
    return model, d["record"]


def main(argv=None) -> None:
    """Train the motif subtree-size network on sizes the plain enumerator
    measures (every root of R-MAT scale-12 graphs, seeds 100-131, k = 5 and
    6) and write it to ``--out``."""
    import argparse
    import time

    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--k", type=int, nargs="+", default=[5, 6])
    ap.add_argument("--seeds", type=int, nargs=2, default=[100, 132])
    ap.add_argument("--scale", type=int, default=12)
    ap.add_argument("--epochs", type=int, default=60)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    X, T = training_set(gpm.GPM_APP_MOTIF, a.k, seeds=range(*a.seeds), scale=a.scale, stream=stream)
    label_s = time.perf_counter() - t0
    model = new_model(0, stream)
    t0 = time.perf_counter()
    train(model, X, T, epochs=a.epochs, batch=4096, lr=3e-3, stream=stream)
    torch.cuda.synchronize()
    record = {"app": "motif", "k": a.k, "graphs": f"R-MAT scale {a.scale}, edge factor 8, seeds "
              f"{a.seeds[0]}-{a.seeds[1] - 1}", "samples": int(X.shape[0]), "epochs": a.epochs,
              "label_s": round(label_s, 1), "train_s": round(time.perf_counter() - t0, 2),
              "first_mse": model.history[0], "final_mse": model.history[-1],
              "device": torch.cuda.get_device_name(0)}
    save(model, a.out, record)
    print(json.dumps(record))


if __name__ == "__main__":
    main()
