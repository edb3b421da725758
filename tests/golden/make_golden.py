"""Write the stored expected counts under tests/golden/ -- calls the oracle only.

Run from the repository root:  python tests/golden/make_golden.py [names...]

Every value written here comes from ``oracle/`` (the plain CPU restatement of
Eq. 1 / Algorithm 4) on the seeded synthetic workloads of
``paper_2212_04551_gb300.graphs``; nothing is read back from the CUDA path.
Root samples are seeded and recorded in the file next to the counts, so the
GPU tests ask the library for exactly the same roots.

Output: one JSON file per workload, ``<name>.json``:
  {"workload": ..., "sha256": <CSR hash>, "cases": [
      {"app": "clique"|"motif", "k": k, "roots": null | [...],
       "order": "id"|"degree",            # clique root order of per-root values
       "total": int, "per_root": [...] | null,
       "patterns": {canonical_code: count} | null}, ...]}
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2212_04551_gb300 import graphs as G  # noqa: E402


def _clique_case(g, k, roots, order):
    t = time.time()
    if roots is None:
        total = O.clique_count(g, k, order=order)
        pr = None
    else:
        total, pr = O.clique_count(g, k, order=order, roots=roots, per_root=True)
        pr = [int(x) for x in pr]
    return {"app": "clique", "k": k, "roots": None if roots is None else [int(r) for r in roots],
            "order": "degree" if order == O.ORDER_DEGREE else "id",
            "total": int(total), "per_root": pr, "patterns": None, "oracle_s": round(time.time() - t, 2)}


def _motif_case(g, k, roots):
    t = time.time()
    if roots is None:
        pats = O.motif_count(g, k)
        pr = None
    else:
        pats, pr = O.motif_count(g, k, roots=roots, per_root=True)
        pr = [int(x) for x in pr]
    return {"app": "motif", "k": k, "roots": None if roots is None else [int(r) for r in roots],
            "order": "id", "total": int(sum(pats.values())), "per_root": pr,
            "patterns": {str(c): int(v) for c, v in sorted(pats.items())},
            "oracle_s": round(time.time() - t, 2)}


def chunglu_roots(g):
    """256 uniform roots plus 64 roots with oriented out-degree in [16, 64]."""
    d = g.degrees()
    e = g.edges()
    du, dv = d[e[:, 0]], d[e[:, 1]]
    fwd = (du < dv) | ((du == dv) & (e[:, 0] < e[:, 1]))
    outdeg = np.bincount(np.where(fwd, e[:, 0], e[:, 1]), minlength=g.n)
    a = G.sample_roots(g.n, 256, seed=11)
    mid = (outdeg >= 16) & (outdeg <= 64)
    b = G.sample_roots(g.n, 64, seed=12, exclude=~mid)
    return np.unique(np.concatenate([a, b])).astype(np.int32)


def rmat_roots(g, k):
    """1,024 seeded roots among vertices whose id is >= 1024 and degree <= 32
    (R-MAT puts its hubs at small ids; every subgraph's root is its smallest
    vertex, so these roots keep the hubs out of their subgraphs)."""
    d = g.degrees()
    ok = (np.arange(g.n) >= 1024) & (d <= 32)
    return G.sample_roots(g.n, 1024, seed=20 + k, exclude=~ok)


def sbm_motif_roots(g):
    return G.sample_roots(g.n, 64, seed=30)


def job(spec):
    name, app, k, roots_kind = spec
    g = G.workload(name)
    if roots_kind is None:
        roots = None
    elif roots_kind == "chunglu":
        roots = chunglu_roots(g)
    elif roots_kind == "rmat":
        roots = rmat_roots(g, k)
    elif roots_kind == "sbm":
        roots = sbm_motif_roots(g)
    else:
        raise KeyError(roots_kind)
    if app == "clique":
        order = O.ORDER_DEGREE if roots is not None else O.ORDER_ID
        return name, _clique_case(g, k, roots, order)
    return name, _motif_case(g, k, roots)


SPECS = {
    "er516": [("er516", "motif", k, None) for k in (3, 4, 5)] + [("er516", "clique", k, None) for k in (3, 4)],
    "sbm2000": [("sbm2000", "clique", k, None) for k in range(3, 13)]
    + [("sbm2000", "motif", 6, "sbm"), ("sbm2000", "motif", 4, None)],
    "rmat16": [("rmat16", "motif", k, "rmat") for k in (5, 6, 7)],
    "chunglu1m": [("chunglu1m", "clique", k, "chunglu") for k in (4, 5, 6, 7, 8)],
}


def main(names):
    O.build()
    specs = [s for n in names for s in SPECS[n]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(specs), os.cpu_count() or 1)) as pool:
        results = pool.map(job, specs, chunksize=1)
    by_name: dict[str, list] = {}
    for name, case in results:
        by_name.setdefault(name, []).append(case)
    for name, cases in by_name.items():
        g = G.workload(name)
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump({"workload": name, "sha256": g.sha256(), "cases": cases}, f, indent=0)
        print(name, [(c["app"], c["k"], c["total"], c["oracle_s"]) for c in cases], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(SPECS))
