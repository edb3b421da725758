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


def _dag_outdeg(g):
    d = g.degrees()
    e = g.edges()
    du, dv = d[e[:, 0]], d[e[:, 1]]
    fwd = (du < dv) | ((du == dv) & (e[:, 0] < e[:, 1]))
    return np.bincount(np.where(fwd, e[:, 0], e[:, 1]), minlength=g.n)


def chunglu_roots(g):
    """320 seeded roots the oracle can finish for k <= 8: 256 uniform roots
    and 64 roots with oriented out-degree in [12, 24], all of degree <= 200
    (the oracle's clique step scans the root's whole adjacency at every node,
    and C(24, 7) bounds a root's 8-cliques)."""
    d = g.degrees()
    outdeg = _dag_outdeg(g)
    ok = (d <= 200) & (outdeg <= 24)
    a = G.sample_roots(g.n, 256, seed=11, exclude=~ok)
    mid = ok & (outdeg >= 12)
    b = G.sample_roots(g.n, 64, seed=12, exclude=~mid)
    return np.unique(np.concatenate([a, b])).astype(np.int32)


def bounded_roots(g, k, count, seed, min_id=0, max_reach=None):
    """Seeded roots whose connected k-sets the oracle can enumerate: walking a
    seeded permutation of the vertices >= min_id, a root r is kept when the
    vertices > r within distance k-1 of r (restricted to vertices > r, the
    only ones a set rooted at r can hold) number at most max_reach, so
    C(reach, k-1) bounds its sets."""
    from math import comb
    if max_reach is None:
        max_reach = {3: 2000, 4: 200, 5: 80, 6: 44, 7: 32}[k]
    rng = np.random.default_rng(seed)
    cand = rng.permutation(np.arange(min_id, g.n))
    ip, ix = g.indptr, g.indices
    out = []
    for r in cand:
        r = int(r)
        seen = {r}
        frontier = [r]
        ok = True
        for _ in range(k - 1):
            nxt = []
            for u in frontier:
                for w in ix[ip[u]:ip[u + 1]]:
                    w = int(w)
                    if w > r and w not in seen:
                        seen.add(w)
                        nxt.append(w)
                        if len(seen) - 1 > max_reach:
                            ok = False
                            break
                if not ok:
                    break
            if not ok:
                break
            frontier = nxt
        if ok and len(seen) > 1 and comb(len(seen) - 1, k - 1) > 0:
            out.append(r)
            if len(out) == count:
                break
    return np.sort(np.array(out, dtype=np.int32))


def rmat_roots(g, k):
    """1,024 seeded bounded roots (see bounded_roots) among ids >= 1024."""
    return bounded_roots(g, k, 1024, seed=20 + k, min_id=1024)


def sbm_motif_roots(g):
    return bounded_roots(g, 6, 32, seed=30, max_reach=400)


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


def chunglu_full_job(chunk):
    """Search-tree instrumentation of the degree-oriented clique enumeration
    to depth 6 over one slice of the roots (every 64th root of the heaviest-
    first order, starting at `chunk`)."""
    g = G.workload("chunglu1m")
    od = _dag_outdeg(g)
    order = np.argsort(-od, kind="stable").astype(np.int32)
    roots = np.ascontiguousarray(order[chunk::64])
    t = time.time()
    r = O.clique_instrument(g, 6, roots=roots)
    return r["nodes"], r["b_alg"], round(time.time() - t, 1)


def write_chunglu_full(pool):
    """Full-size clique counts k = 4..6 of chunglu1m (the benchmark's
    workload) and the list-merge bytes B_alg of the depth-6 search, summed
    over a partition of the roots."""
    res = pool.map(chunglu_full_job, range(64), chunksize=1)
    nodes = [sum(r[0][s] for r in res) for s in range(7)]
    g = G.workload("chunglu1m")
    out = {"workload": "chunglu1m", "sha256": g.sha256(), "k_max": 6,
           "cliques": {str(s): int(nodes[s]) for s in range(1, 7)},
           "b_alg_depth6": int(sum(r[1] for r in res)),
           "oracle_s_max_chunk": max(r[2] for r in res)}
    with open(os.path.join(HERE, "chunglu1m_full.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("chunglu1m_full", out["cliques"], out["b_alg_depth6"], flush=True)


def chunglu_heaviest_first(g):
    """Roots of chunglu1m, heaviest oriented out-degree first (stable)."""
    return np.argsort(-_dag_outdeg(g), kind="stable").astype(np.int32)


def chunglu_k78_job(spec):
    """Bitset-route clique counts of one root slice: (k, slice of the
    heaviest-first order).  k = 7 slices are every 64th root starting at c;
    k = 8 slices cut the 1/64 sample (every 64th root from 0) 32 ways."""
    k, part = spec
    g = G.workload("chunglu1m")
    order = chunglu_heaviest_first(g)
    roots = order[part::64] if k == 7 else order[0::64][part::32]
    roots = np.ascontiguousarray(roots)
    t = time.time()
    counts, pr = O.clique_count_bits(g, k, roots=roots, per_root=True)
    return spec, roots, counts, pr, round(time.time() - t, 1)


def write_chunglu_k78(pool):
    """chunglu1m clique counts at k = 7 over every root (totals per size and
    a hash of the per-root 6- and 7-clique counts, indexed by vertex id) and
    at k = 8 over the seeded 1/64 sample of the heaviest-first order (every
    64th root from the heaviest; per-root 7- and 8-clique counts), by the
    oracle's bitset route."""
    import hashlib
    specs = [(8, j) for j in range(32)] + [(7, c) for c in range(64)]
    res = pool.map(chunglu_k78_job, specs, chunksize=1)
    g = G.workload("chunglu1m")
    tot7 = [0] * 8
    pr7 = np.zeros((g.n, 8), dtype=np.uint64)
    samp = {}
    tot8 = [0] * 9
    secs = {7: 0.0, 8: 0.0}
    for (k, part), roots, counts, pr, t in res:
        secs[k] = max(secs[k], t)
        if k == 7:
            for s in range(8):
                tot7[s] += counts[s]
            pr7[roots] = pr
        else:
            for s in range(9):
                tot8[s] += counts[s]
            for r, row in zip(roots.tolist(), pr):
                samp[r] = (int(row[7]), int(row[8]))
    order = chunglu_heaviest_first(g)
    sample = order[0::64]
    out = {"workload": "chunglu1m", "sha256": g.sha256(), "route": "bits",
           "k7_all_roots": {"cliques": {str(s): int(tot7[s]) for s in range(1, 8)},
                            "per_root_sha256": {str(s): hashlib.sha256(np.ascontiguousarray(pr7[:, s], dtype="<u8")
                                                                       .tobytes()).hexdigest() for s in (6, 7)},
                            "oracle_s_max_slice": secs[7]},
           "k8_sample": {"rule": "every 64th root of the heaviest-first order (stable sort by oriented "
                                 "out-degree, descending), starting at the heaviest",
                         "n_roots": int(sample.shape[0]),
                         "cliques": {str(s): int(tot8[s]) for s in range(1, 9)},
                         "per_root": [[int(r), samp[int(r)][0], samp[int(r)][1]] for r in sample
                                      if samp[int(r)][0]],
                         "oracle_s_max_slice": secs[8]}}
    with open(os.path.join(HERE, "chunglu1m_k78.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("chunglu1m_k78", out["k7_all_roots"]["cliques"], out["k8_sample"]["cliques"], secs, flush=True)


def rmat_bench_roots(g):
    """The 512 seeded roots the learned-scheduling comparison uses: ids >=
    1024 with degree <= 32 (seed 25)."""
    d = g.degrees()
    ok = (np.arange(g.n) >= 1024) & (d <= 32)
    return G.sample_roots(g.n, 512, seed=25, exclude=~ok)


def esu_job(spec):
    """ESU-route motif counts of one slice of the roots (every 64th root of
    the given root list, heaviest degree first, starting at `part`)."""
    name, k, roots_kind, part = spec
    g = G.workload(name)
    if roots_kind == "all":
        roots = np.argsort(-g.degrees(), kind="stable").astype(np.int32)
    else:
        roots = rmat_bench_roots(g)
    mine = np.ascontiguousarray(roots[part::64]).astype(np.int32)
    t = time.time()
    pats, pr = O.motif_count(g, k, roots=mine, per_root=True, method="esu")
    return spec, mine.tolist(), pats, [int(x) for x in pr], round(time.time() - t, 1)


FULL_SPECS = {
    "rmat16_full": [("rmat16", 4, "all"), ("rmat16", 5, "bench")],
    "sbm2000_full": [("sbm2000", 5, "all"), ("sbm2000", 6, "all")],
}


def write_full(pool, fname):
    """Motif counts over every root (or the 512-root benchmark sample) by the
    oracle's ESU route, summed over 64 root slices."""
    specs = [(name, k, kind, part) for name, k, kind in FULL_SPECS[fname] for part in range(64)]
    res = pool.map(esu_job, specs, chunksize=1)
    cases = []
    for name, k, kind in FULL_SPECS[fname]:
        pats, per_root = {}, {}
        secs = 0.0
        for spec, mine, p, pr, t in res:
            if spec[:3] != (name, k, kind):
                continue
            for c, v in p.items():
                pats[c] = pats.get(c, 0) + v
            per_root.update(zip(mine, pr))
            secs = max(secs, t)
        g = G.workload(name)
        roots = None if kind == "all" else [int(r) for r in rmat_bench_roots(g)]
        cases.append({"app": "motif", "k": k, "roots": roots, "order": "id",
                      "total": int(sum(pats.values())),
                      "per_root": None if roots is None else [per_root[r] for r in roots],
                      "patterns": {str(c): int(v) for c, v in sorted(pats.items())},
                      "oracle_s": secs, "route": "esu"})
    name = FULL_SPECS[fname][0][0]
    with open(os.path.join(HERE, f"{fname}.json"), "w") as f:
        json.dump({"workload": name, "sha256": G.workload(name).sha256(), "cases": cases}, f, indent=0)
    print(fname, [(c["k"], c["total"], c["oracle_s"]) for c in cases], flush=True)


RMAT_BANDS = [(1, 4), (4, 16), (16, 64), (64, 256), (256, 1024), (1024, 1 << 30)]
RMAT_PER_BAND = 16
RMAT_ROOT_LIMIT_S = 150


def rmat_strat_candidates(g, k):
    """Candidate roots of the stratified rmat16 sample at size k: up to 16
    seeded roots from each band of up-degree (neighbours above the root, the
    size of its first extension set): 1-3, 4-15, 16-63, 64-255, 256-1023,
    1024 and more."""
    ip, ix = g.indptr, g.indices
    src = np.repeat(np.arange(g.n), np.diff(ip))
    up = np.bincount(src[ix > src], minlength=g.n)
    rng = np.random.default_rng(60 + k)
    out = []
    for lo, hi in RMAT_BANDS:
        pool = np.nonzero((up >= lo) & (up < hi))[0]
        pick = rng.choice(pool, size=min(RMAT_PER_BAND, pool.shape[0]), replace=False) if pool.shape[0] else []
        out.extend((int(lo), int(r)) for r in sorted(int(x) for x in pick))
    return out


def one_root(name, k, r):
    """Child-process mode: the ESU-route motif counts of one root, as JSON."""
    g = G.workload(name)
    pats, pr = O.motif_count(g, k, roots=np.array([r], dtype=np.int32), per_root=True, method="esu")
    print(json.dumps({"patterns": {str(c): int(v) for c, v in pats.items()}, "total": int(pr[0])}))


def write_rmat16_strat():
    """rmat16 motif counts at k = 5, 6, 7 on stratified root samples (see
    rmat_strat_candidates): every candidate runs through the oracle's ESU
    route in its own process, and a root whose run takes longer than
    RMAT_ROOT_LIMIT_S seconds is left out (listed under "dropped") -- so the
    sample holds the heaviest roots the oracle can finish."""
    import subprocess
    g = G.workload("rmat16")
    tasks = [(k, band, r) for k in (5, 6, 7) for band, r in rmat_strat_candidates(g, k)]
    tasks.sort(key=lambda t: (t[1], t[0]))          # light bands first

    def run(task):
        k, band, r = task
        t = time.time()
        try:
            p = subprocess.run([sys.executable, os.path.abspath(__file__), "--one-root", "rmat16", str(k), str(r)],
                               capture_output=True, text=True, timeout=RMAT_ROOT_LIMIT_S)
        except subprocess.TimeoutExpired:
            return task, None, round(time.time() - t, 1)
        if p.returncode != 0:
            raise RuntimeError(p.stderr)
        return task, json.loads(p.stdout.strip().splitlines()[-1]), round(time.time() - t, 1)

    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 1) - 1)) as ex:
        res = list(ex.map(run, tasks))
    cases = []
    for k in (5, 6, 7):
        done = sorted((t[2], out, secs) for t, out, secs in res if t[0] == k and out is not None)
        dropped = sorted(t[2] for t, out, _ in res if t[0] == k and out is None)
        pats: dict = {}
        for _, out, _ in done:
            for c, v in out["patterns"].items():
                pats[c] = pats.get(c, 0) + v
        cases.append({"app": "motif", "k": k, "roots": [r for r, _, _ in done],
                      "per_root": [out["total"] for _, out, _ in done],
                      "total": sum(out["total"] for _, out, _ in done),
                      "patterns": dict(sorted(pats.items(), key=lambda kv: int(kv[0]))),
                      "dropped": dropped, "oracle_s_max_root": max((s for _, _, s in done), default=0.0),
                      "rule": f"up to {RMAT_PER_BAND} seeded roots (seed {60 + k}) per up-degree band "
                              f"{[b for b, _ in RMAT_BANDS]}, keeping those the oracle's ESU route "
                              f"finishes within {RMAT_ROOT_LIMIT_S} s"})
    with open(os.path.join(HERE, "rmat16_strat.json"), "w") as f:
        json.dump({"workload": "rmat16", "sha256": g.sha256(), "route": "esu", "cases": cases}, f, indent=0)
    print("rmat16_strat", [(c["k"], len(c["roots"]), len(c["dropped"]), c["total"]) for c in cases], flush=True)


def ba_graphs():
    """48 seeded graph indices of the 4,096-graph Barabasi-Albert batch."""
    rng = np.random.default_rng(40)
    return sorted(int(i) for i in rng.choice(4096, 48, replace=False))


def ba_job(idx):
    """Per-graph 4-clique count and 5-vertex motif counts of one batch graph."""
    g = G.workload("ba4096")[idx]
    t = time.time()
    c4 = int(O.clique_count(g, 4))
    m5 = {str(c): int(v) for c, v in sorted(O.motif_count(g, 5).items())}
    return idx, c4, m5, round(time.time() - t, 2)


def ba_hash():
    import hashlib
    h = hashlib.sha256()
    for g in G.workload("ba4096"):
        h.update(g.sha256().encode())
    return h.hexdigest()


def write_ba(pool):
    idx = ba_graphs()
    res = pool.map(ba_job, idx, chunksize=1)
    out = {"workload": "ba4096", "sha256": ba_hash(), "graphs": [r[0] for r in res],
           "clique4": [r[1] for r in res], "motif5": [r[2] for r in res]}
    with open(os.path.join(HERE, "ba4096.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("ba4096", len(res), "graphs, oracle s max", max(r[3] for r in res), flush=True)


SPECS = {
    "er516": [("er516", "motif", k, None) for k in (3, 4, 5)] + [("er516", "clique", k, None) for k in (3, 4)],
    "sbm2000": [("sbm2000", "clique", k, None) for k in range(3, 13)]
    + [("sbm2000", "motif", 6, "sbm"), ("sbm2000", "motif", 4, None)],
    "rmat16": [("rmat16", "motif", k, "rmat") for k in (5, 6, 7)],
    "chunglu1m": [("chunglu1m", "clique", k, "chunglu") for k in (4, 5, 6, 7, 8)],
}


def main(names):
    O.build()
    if "rmat16_strat" in names:
        write_rmat16_strat()
        names = [n for n in names if n != "rmat16_strat"]
    ctx = mp.get_context("spawn")
    if "ba4096" in names:
        with ctx.Pool(os.cpu_count() or 1) as pool:
            write_ba(pool)
        names = [n for n in names if n != "ba4096"]
    if "chunglu1m_k78" in names:
        with ctx.Pool(max(1, (os.cpu_count() or 1) - 1)) as pool:
            write_chunglu_k78(pool)
        names = [n for n in names if n != "chunglu1m_k78"]
    if "chunglu1m_full" in names:
        with ctx.Pool(os.cpu_count() or 1) as pool:
            write_chunglu_full(pool)
        names = [n for n in names if n != "chunglu1m_full"]
    for fname in [n for n in names if n in FULL_SPECS]:
        with ctx.Pool(os.cpu_count() or 1) as pool:
            write_full(pool, fname)
    names = [n for n in names if n not in FULL_SPECS]
    specs = [s for n in names for s in SPECS[n]]
    if not specs:
        return
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
    if sys.argv[1:2] == ["--one-root"]:
        one_root(sys.argv[2], int(sys.argv[3]), int(sys.argv[4]))
        sys.exit(0)
    main(sys.argv[1:] or list(SPECS) + ["ba4096", "chunglu1m_full", "chunglu1m_k78", "rmat16_strat"]
         + list(FULL_SPECS))
