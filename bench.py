"""Benchmark: enumerated subgraphs/s on one GB300 (bit-exact counts).

Default workload (the plain method at scale): k-clique counting on the
Chung-Lu power-law graph (n = 1,000,000, average degree 16, exponent 2.1,
expected degrees capped at 20,000, seed 1), degree-ordered, int32 CSR.  One
step = one enumeration that counts every clique size 4..7
(gpm_clique_count_range), with the graph already resident in HBM.  The
configuration's full range 4..8 is one enumeration of about half a minute:
it is timed once, beside the steps, as the ``k4_8`` entry.

Beside the headline the line carries one timed, oracle-checked entry per
workload of the method (``configs``): 4-vertex motifs on a 516-vertex
Erdos-Renyi graph (plain call and CUDA-graph replay), 5-vertex motifs over
every root of an R-MAT scale-16 graph (plain vs learned scheduling, plus
6- and 7-vertex motifs on a stratified root sample), 4,096 small
Barabasi-Albert graphs (batched launch vs the plain kernel on their union
vs one plain call per graph), and deep cliques plus 6-vertex motifs on a
stochastic block model graph (plain vs learned).  Then the load-balancing
and DM_DFS ablations and subgraph listing through the host ring
(``listing``: records per second to a counting consumer).  ``--full`` adds
the long comparisons (DM_DFS at k = 5, no balancing on the 7-cliques).

Printed: one JSON line (rank 0) with the metric, the device-timed value,
the end-to-end value through the C ABI with host buffers (graph creation
from host CSR + counting + result read-back inside the timed region), the
roofline of the dominant kernel, SM clocks sampled during the timed region,
and the CPU oracle on a stratified root sample of the same workload, run on
every host core.

``--impl reference`` times the CPU oracle alone on such samples (the
reference arm for this method is the plain CPU restatement of the paper's
enumeration).

Multi-GPU (torchrun, N ranks): the roots are split round-robin over the
ranks -- every clique has exactly one root -- and the per-rank counts are
summed on the host; value = all subgraphs / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from math import comb

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "enumerated subgraphs/s on 1 GB300 (bit-exact counts), learned/batched vs plain"
UNIT = "subgraphs/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpm", choices=["gpm", "reference"])
    ap.add_argument("--k-lo", type=int, default=4)
    ap.add_argument("--k-hi", type=int, default=7)
    ap.add_argument("--cpu-stride", type=int, default=512,
                    help="oracle sample: every this-many-th root of the heaviest-first order")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k8", action="store_true", help="skip the timed k = 4..8 enumeration")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-workload entries")
    ap.add_argument("--full", action="store_true",
                    help="also the long comparisons: DM_DFS at k = 5, no balancing on chunglu1m 7-cliques")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run one small launch of a kernel (for ncu captures) and exit")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# The clique kernel's unit of work is one 32-bit candidate-word operation:
# AND of a candidate word with an adjacency-row word, POPC, accumulate.  Its
# peak is set by the population-count rate: 16 results per clock per SM
# (the integer-intrinsic throughput of the CUDA arithmetic-instruction table)
# x 152 SMs x the maximum SM clock.
POPC_PER_CLK_PER_SM = 16
# Instruction issue: 4 schedulers per SM, one warp instruction each per clock.
ISSUE_PER_CLK_PER_SM = 4


def kernel_source_hash(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2212_04551_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_launch(summary: str, src_hash: str, units_now: float) -> dict:
    """Per-launch counters of the same launch from a committed ncu summary
    (profiles/<summary>: DRAM bytes, warp instructions executed), or {} when
    the kernel source changed since or the launch differs (its exact
    word-operation count identifies it)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return {}
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != src_hash:
        return {}
    try:
        u = float(kv["units_per_launch"])
        out = {"dram_bytes": float(kv["dram_bytes_per_launch"]), "warp_inst": float(kv["warp_inst_per_launch"])}
    except (KeyError, ValueError):
        return {}
    return out if u > 0 and abs(units_now - u) <= 1e-6 * u else {}


def golden(name: str):
    """A stored oracle result under tests/golden/ (written by make_golden.py
    from the oracle only), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def oracle_clique_totals(g) -> dict:
    """Full-size clique totals of chunglu1m per size, from the stored oracle
    runs over every root (k <= 6: list route; k = 7: bitset route)."""
    out = {}
    for name, key in (("chunglu1m_full", None), ("chunglu1m_k78", "k7_all_roots")):
        d = golden(name)
        if d is None or d["sha256"] != g.sha256():
            continue
        src = d["cliques"] if key is None else d[key]["cliques"]
        for s, v in src.items():
            out[int(s)] = int(v)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dag_out_degrees(g) -> np.ndarray:
    d = g.degrees()
    e = g.edges()
    du, dv = d[e[:, 0]], d[e[:, 1]]
    fwd = (du < dv) | ((du == dv) & (e[:, 0] < e[:, 1]))
    return np.bincount(np.where(fwd, e[:, 0], e[:, 1]), minlength=g.n)


def heaviest_first(g) -> np.ndarray:
    return np.argsort(-dag_out_degrees(g), kind="stable").astype(np.int32)


# ---------------------------------------------------------------- CPU oracle

def cpu_baseline(g, k_lo, k_hi, stride, offset=0, cores=None):
    """The oracle (its bitset clique route, every size k_lo..k_hi in one
    pass) on a stratified root sample of the same workload -- every
    ``stride``-th root of the heaviest-first order from ``offset``, so heavy
    and light roots are mixed as in the full run -- spread over the host
    cores by threads (the oracle's C code runs without the interpreter lock).
    Returns (subgraphs/s, description, cores used, subgraphs, seconds)."""
    from oracle import oracle as O
    O.build()
    roots = heaviest_first(g)[offset::stride]
    cores = cores or os.cpu_count() or 1
    chunks = [np.ascontiguousarray(roots[i::cores * 4]) for i in range(cores * 4)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(lambda r: O.clique_count_bits(g, k_hi, roots=r), chunks))
    el = time.perf_counter() - t0
    found = sum(sum(c[k] for k in range(k_lo, k_hi + 1)) for c in res)
    desc = (f"oracle clique k={k_lo}..{k_hi} (bitset route, one pass) on every {stride}th root of the "
            f"heaviest-first order from {offset} ({roots.shape[0]} roots, {el:.1f} s on {cores} threads)")
    return found / el, desc, cores, found, el


def timed(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def by_code(k, counts) -> dict:
    from paper_2212_04551_gb300 import gpm
    return {str(gpm.gpm_motif_pattern(k, p)): int(x) for p, x in enumerate(counts) if x}


def dominating(k, code) -> int:
    adj = [[False] * k for _ in range(k)]
    for i in range(1, k):
        for j in range(i):
            if (code >> (i * (i - 1) // 2 + j)) & 1:
                adj[i][j] = adj[j][i] = True
    return sum(1 for v in range(k) if all(adj[v][u] for u in range(k) if u != v))


def motif_stats(dg) -> dict:
    from paper_2212_04551_gb300 import gpm
    st = gpm.gpm_get_stats(dg)
    return {"kernel_ms": st["kernel_ms"], "donations": int(st["donations"]), "units": int(st["units_done"]),
            "idle_warp_frac": st["idle_warp_frac"], "adjacency_entries": int(st["word_ops"]),
            "grid": [int(st["grid_blocks"]), int(st["warps_per_block"])]}


_L2 = {}


def l2_peaks() -> dict:
    """The GB300's L2 read bandwidth, measured here by the library
    (gpm_measure_l2): 64 MB streamed with coalesced 16-byte loads, and the
    same buffer read one 32-byte sector at a time at random."""
    from paper_2212_04551_gb300 import gpm
    if not _L2:
        _L2["stream_gbs"] = max(gpm.gpm_measure_l2(64 << 20, 0, 20) for _ in range(3))
        _L2["sector_gbs"] = max(gpm.gpm_measure_l2(64 << 20, 1, 20) for _ in range(3))
    return dict(_L2)


def motif_roofline(arm: dict) -> dict:
    """The motif kernel against L2: every scanned adjacency entry moves 4 B
    of index (coalesced) and selects one mark byte at a random place, which
    costs one 32-byte L2 sector; achieved = entries x 36 B / kernel time,
    against the measured random-sector L2 bandwidth.  (Algorithmic bytes, 4
    + 1 per entry, are given beside it.)"""
    pk = l2_peaks()
    s = arm["kernel_ms"] / 1000.0
    e = float(arm["adjacency_entries"])
    ach = e * 36.0 / s / 1e9
    return {"bound": "l2", "kernel": "k_motif", "achieved": ach, "peak": pk["sector_gbs"], "unit": "GB/s",
            "frac": ach / pk["sector_gbs"], "peak_kind": "measured random 32-byte sector reads (gpm_measure_l2)",
            "bytes_per_entry": 36, "algorithmic_gbs": e * 5.0 / s / 1e9,
            "l2_stream_peak_gbs": pk["stream_gbs"], "units_per_launch": e}


# ---------------------------------------------------------- learned scheduler

class Learned:
    """The subtree-size MLP and an untrained copy (the ablation).  The trained
    network is the one shipped with the package -- trained by the library's
    own kernels on sizes the plain enumerator measured (motif counting, k = 5
    and 6, every root of the 32 R-MAT scale-12 graphs of seeds 100-131; its
    record rides along) -- or, when that file is absent, one trained here on
    the k = 5 sizes only (the k = 6 labels take minutes)."""

    def __init__(self, stream, epochs=40):
        from paper_2212_04551_gb300 import gpm
        from paper_2212_04551_gb300 import learned as L
        self.stream = stream
        self.untrained = L.new_model(0, stream)
        if os.path.exists(L.WEIGHTS):
            self.model, rec = L.load(L.WEIGHTS, stream)
            self.info = {"source": os.path.relpath(L.WEIGHTS, ROOT), **rec}
            return
        t0 = time.perf_counter()
        X, T = L.training_set(gpm.GPM_APP_MOTIF, (5,), seeds=range(100, 132), scale=12, stream=stream)
        label_s = time.perf_counter() - t0
        self.model = L.new_model(0, stream)
        t0 = time.perf_counter()
        L.train(self.model, X, T, epochs=epochs, batch=4096, lr=3e-3, stream=stream)
        import torch
        torch.cuda.synchronize()
        self.info = {"source": "trained in this run", "k": [5], "samples": int(X.shape[0]), "epochs": epochs,
                     "label_s": round(label_s, 2), "train_s": round(time.perf_counter() - t0, 2),
                     "first_mse": self.model.history[0], "final_mse": self.model.history[-1]}

    def compare(self, dg, g, k, roots=None, reps=1, arms=("plain", "learned", "untrained"), static=False):
        """Plain (heaviest degree first, donation) against the learned and
        untrained schedules on the same root set; counts must agree."""
        from scipy.stats import spearmanr

        from paper_2212_04551_gb300 import gpm
        from paper_2212_04551_gb300 import learned as L
        feats = L.features(dg, g.n, k)
        preds = {"learned": L.predict(self.model, feats, self.stream),
                 "untrained": L.predict(self.untrained, feats, self.stream)}
        n_roots = g.n if roots is None else len(roots)
        out, ref, sizes = {}, None, None
        warps = 4864
        for donate in ((1, 0) if static else (1,)):
            gpm.gpm_set_config(dg, donate=donate)
            tag = "donation" if donate else "static"
            res = {}
            for name in arms:
                if name == "plain":
                    gpm.gpm_sched_from_scores(dg, gpm.GPM_APP_MOTIF, None, roots, 0, 0)
                    plan = {"split_roots": 0, "chunks": 0}
                else:
                    plan = L.schedule(dg, gpm.GPM_APP_MOTIF, preds[name], roots, warps=warps)
                times = []
                for _ in range(reps):
                    (c, pr), ms = timed(lambda: gpm.gpm_count_scheduled(dg, gpm.GPM_APP_MOTIF, k, n_roots=n_roots,
                                                                        per_root=True), self.stream)
                    times.append(ms)
                if ref is None:
                    ref, sizes = c, pr
                assert np.array_equal(c, ref), f"{name} schedule changed the counts"
                ms = statistics.median(times)
                res[name] = {"ms": ms, "subgraphs_per_s": int(ref.sum()) / (ms / 1000.0), **motif_stats(dg), **plan}
                if name == "plain":
                    warps = res[name]["grid"][0] * res[name]["grid"][1]
            if "plain" in res and "learned" in res:
                res["speedup_learned_vs_plain"] = res["plain"]["ms"] / res["learned"]["ms"]
            if "plain" in res and "untrained" in res:
                res["speedup_untrained_vs_plain"] = res["plain"]["ms"] / res["untrained"]["ms"]
            out[tag] = res
        gpm.gpm_set_config(dg, donate=1)
        sel = np.arange(g.n) if roots is None else np.asarray(roots)
        meas = np.log1p(sizes.astype(np.float64))
        out["spearman_trained"] = float(spearmanr(preds["learned"].cpu().numpy()[sel], meas).statistic)
        out["spearman_untrained"] = float(spearmanr(preds["untrained"].cpu().numpy()[sel], meas).statistic)
        out["spearman_degree"] = float(spearmanr(g.degrees()[sel], meas).statistic)
        return out, ref, sizes


# ------------------------------------------------------------ per-workload

def config_er516(stream) -> dict:
    """4-vertex motifs of the 516-vertex Erdos-Renyi graph: the plain call
    (median of 20) and one persistent launch captured in a CUDA graph,
    replayed 100 times (time / 100)."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    g = G.workload("er516")
    dg = gpm.graph_from_csr(g, stream=stream)
    c = gpm.gpm_motif_count(dg, 4)
    kms, wall = [], []
    for _ in range(20):
        t0 = time.perf_counter()
        gpm.gpm_motif_count(dg, 4)
        wall.append((time.perf_counter() - t0) * 1000)
        kms.append(gpm.gpm_get_stats(dg)["kernel_ms"])
    b = gpm.batch_from_graphs([g], stream=stream)
    _, bm = gpm.gpm_batch_count(b, 0, 4)
    _, ms100 = timed(lambda: [gpm.gpm_batch_count(b, 0, 4) for _ in range(100)], stream)
    gd = golden("er516")
    want = next(cs["patterns"] for cs in gd["cases"] if cs["app"] == "motif" and cs["k"] == 4) if gd else None
    total = int(c.sum())
    b.close()
    dg.close()
    return {"workload": "er516 motif k=4 (n=516, m=1,200, seed 0)", "subgraphs": total,
            "plain_kernel_ms": statistics.median(kms), "plain_call_ms": statistics.median(wall),
            "plain_subgraphs_per_s": total / (statistics.median(wall) / 1000.0),
            "graph_replay_ms": ms100 / 100.0, "graph_replay_subgraphs_per_s": total / (ms100 / 100.0 / 1000.0),
            "oracle_parity": (by_code(4, c) == want and by_code(4, bm[0]) == want) if want else None}


def config_rmat16(stream, learned: Learned, full: bool = False) -> dict:
    """5-vertex motifs over every root of R-MAT scale 16 (hub of degree 6,444
    at id 0), plain and learned; pinned by the star identity
    sum_p dom(p) count_p = sum_v C(d(v), 4).  6- and 7-vertex motifs on the
    stratified root samples stored beside the oracle's counts."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    g = G.workload("rmat16")
    dg = gpm.graph_from_csr(g, stream=stream)
    d = g.degrees()
    res = {"workload": "rmat16 motif k=5 every root (R-MAT scale 16, edge factor 8, seed 2)"}
    cmp5, c5, _ = learned.compare(dg, g, 5, None, reps=1, arms=("plain", "learned"))
    lhs = sum(dominating(5, gpm.gpm_motif_pattern(5, p)) * int(x) for p, x in enumerate(c5))
    res["k5_all_roots"] = {"subgraphs": int(c5.sum()), **cmp5,
                           "star_identity": lhs == sum(comb(int(x), 4) for x in d),
                           "roofline": motif_roofline(cmp5["donation"]["plain"])}
    gs = golden("rmat16_strat")
    if gs is not None and gs["sha256"] == g.sha256():
        for case in gs["cases"]:
            k, roots = case["k"], np.array(case["roots"], dtype=np.int32)
            cmp, c, pr = learned.compare(dg, g, k, roots, reps=1, static=False)
            res[f"k{k}_sample"] = {"roots": len(roots), "sample": case["rule"], "subgraphs": int(c.sum()), **cmp,
                                   "oracle_parity": by_code(k, c) == case["patterns"]
                                   and [int(x) for x in pr] == case["per_root"]}
    dg.close()
    return res


def config_ba4096(stream, reps: int = 5) -> dict:
    """4,096 Barabasi-Albert graphs, per-graph 4-clique and 5-motif counts:
    one autotuned, CUDA-graph-captured persistent launch, against the plain
    kernel on the same graphs packed as one disjoint union (one clique call
    + one motif call: the same subgraphs, but no per-graph results), and
    against one plain call per graph (warmed, median of 3 passes)."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    gs = list(G.workload("ba4096"))
    b = gpm.batch_from_graphs(gs, stream=stream)
    t0 = time.perf_counter()
    best, _ = gpm.gpm_batch_autotune(b, 4, 5, reps=3)
    tune_s = time.perf_counter() - t0
    cc, mc = gpm.gpm_batch_count(b, 4, 5)
    times = []
    for _ in range(reps):
        _, ms = timed(lambda: gpm.gpm_batch_count(b, 4, 5), stream)
        times.append(ms)
    total = int(cc.sum()) + int(mc.sum())
    parity = None
    gd = golden("ba4096")
    if gd is not None:
        parity = all(int(cc[i]) == c4 and by_code(5, mc[i]) == m5
                     for i, c4, m5 in zip(gd["graphs"], gd["clique4"], gd["motif5"]))
    t_b = statistics.median(times)
    idle_b = gpm.gpm_batch_get_stats(b)["idle_warp_frac"]
    # the plain kernel on the disjoint union of all 4,096 graphs
    u = G.disjoint_union(*gs)
    du = gpm.graph_from_csr(u, stream=stream)
    def union():
        return gpm.gpm_clique_count(du, 4), gpm.gpm_motif_count(du, 5)
    union()
    tu = []
    for _ in range(reps):
        (uc, um), ms = timed(union, stream)
        tu.append(ms)
    assert uc == int(cc.sum()) and np.array_equal(um, mc.sum(axis=0)), "union counts differ from the batch"
    du.close()
    # one plain call per graph (graphs resident), warmed
    dgs = [gpm.graph_from_csr(x, stream=stream) for x in gs]
    def loop():
        c = np.array([gpm.gpm_clique_count(d, 4) for d in dgs], dtype=np.uint64)
        m = np.stack([gpm.gpm_motif_count(d, 5) for d in dgs])
        return c, m
    loop()
    tl = []
    for _ in range(3):
        (pc, pm), ms = timed(loop, stream)
        tl.append(ms)
    assert np.array_equal(pc, cc) and np.array_equal(pm, mc), "batched counts differ from per-graph counts"
    for d in dgs:
        d.close()
    b.close()
    t_u, t_l = statistics.median(tu), statistics.median(tl)
    return {"workload": "ba4096: 4,096 BA graphs (n~U[20,400], m_a~U[2,6], seed 3), clique k=4 + motif k=5 per graph",
            "graphs": len(gs), "subgraphs": total,
            "batched_ms": t_b, "batched_subgraphs_per_s": total / (t_b / 1000.0),
            "plain_union_ms": t_u, "plain_union_subgraphs_per_s": total / (t_u / 1000.0),
            "plain_per_graph_ms": t_l, "plain_per_graph_call_ms": t_l / (2 * len(gs)),
            "speedup_vs_plain_union": t_u / t_b, "speedup_vs_plain_per_graph": t_l / t_b,
            "autotuned": best, "autotune_s": round(tune_s, 1), "batched_idle_warp_frac": idle_b,
            "oracle_parity_48_graphs": parity}


def config_sbm2000(stream, learned: Learned) -> dict:
    """Stochastic block model (2,000 vertices, 20 blocks): every clique size
    6..12 from one enumeration, and 6-vertex motifs plain vs learned."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    g = G.workload("sbm2000")
    dg = gpm.graph_from_csr(g, stream=stream)
    cr = gpm.gpm_clique_count_range(dg, 6, 12)
    kms = []
    for _ in range(3):
        cr = gpm.gpm_clique_count_range(dg, 6, 12)
        kms.append(gpm.gpm_get_stats(dg)["kernel_ms"])
    gd = golden("sbm2000")
    want = {cs["k"]: cs["total"] for cs in gd["cases"] if cs["app"] == "clique" and cs["roots"] is None} if gd else {}
    res = {"workload": "sbm2000 (n=2,000, 20 blocks, p_in 0.5, p_out 0.01, seed 4)",
           "clique_6_12": {"counts": {str(k): int(c) for k, c in zip(range(6, 13), cr)},
                           "kernel_ms": statistics.median(kms),
                           "subgraphs_per_s": sum(int(c) for c in cr) / (statistics.median(kms) / 1000.0),
                           "oracle_parity": all(int(c) == want.get(k) for k, c in zip(range(6, 13), cr))}}
    cmp6, c6, _ = learned.compare(dg, g, 6, None, reps=1, arms=("plain", "learned", "untrained"))
    gf = golden("sbm2000_full")
    want6 = next((cs["patterns"] for cs in gf["cases"] if cs["k"] == 6 and cs["roots"] is None), None) if gf else None
    res["motif6"] = {"subgraphs": int(c6.sum()), **cmp6, "oracle_parity": by_code(6, c6) == want6 if want6 else None,
                     "roofline": motif_roofline(cmp6["donation"]["plain"])}
    dg.close()
    return res


def balancing_ablation(stream, full: bool = False) -> dict:
    """Load balancing on the same kernels and GB300 (the paper's Section
    4.3.5 and Table optimizations-performance, on this hardware): the
    in-kernel hand-off (the plain method's default), the paper's
    host-monitored stop / redistribute / restart (thresholds 40 % for
    cliques and 10 % for motifs, the paper's best), and no balancing at
    all.  Workloads: chunglu1m 7-cliques (the headline's deepest size) and
    sbm2000 5-motifs."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    out = {}
    for name, app, k, th in (("chunglu1m", gpm.GPM_APP_CLIQUE, 7, 0.4), ("sbm2000", gpm.GPM_APP_MOTIF, 5, 0.1)):
        g = G.workload(name)
        dg = gpm.graph_from_csr(g, stream=stream)
        res = {}
        if app == gpm.GPM_APP_CLIQUE:
            ref, ms = timed(lambda: gpm.gpm_clique_count(dg, k), stream)
            ref = np.array([ref], dtype=np.uint64)
        else:
            ref, ms = timed(lambda: gpm.gpm_motif_count(dg, k), stream)
        st = gpm.gpm_get_stats(dg)
        res["in_kernel_handoff"] = {"ms": ms, "kernel_ms": st["kernel_ms"], "idle_warp_frac": st["idle_warp_frac"],
                                    "handoffs": int(st["donations"])}
        t0 = time.perf_counter()
        c, mst = gpm.gpm_count_monitored(dg, app, k, th)
        res["host_monitored"] = {"ms": (time.perf_counter() - t0) * 1000.0, "threshold": th, **mst,
                                 "same_counts": bool(np.array_equal(c, ref))}
        res["speedup_handoff_vs_monitored"] = res["host_monitored"]["ms"] / res["in_kernel_handoff"]["ms"]
        if full or app != gpm.GPM_APP_CLIQUE:
            gpm.gpm_set_config(dg, donate=0)
            c = gpm.gpm_clique_count(dg, k) if app == gpm.GPM_APP_CLIQUE else gpm.gpm_motif_count(dg, k)
            st = gpm.gpm_get_stats(dg)
            res["none"] = {"kernel_ms": st["kernel_ms"], "idle_warp_frac": st["idle_warp_frac"],
                           "same_counts": bool(np.array_equal(np.ravel(c), np.ravel(ref)))}
            res["speedup_handoff_vs_none"] = res["none"]["kernel_ms"] / res["in_kernel_handoff"]["kernel_ms"]
        out[f"{name}_{'clique' if app == gpm.GPM_APP_CLIQUE else 'motif'}{k}"] = res
        dg.close()
    return out


def dm_dfs_ablation(stream, full: bool = False) -> dict:
    """The paper's DM_DFS baseline (one thread per root, sorted-list merges,
    no balancing) against the warp-centric bitmap kernel with hand-offs, on
    chunglu1m cliques k = 4 and 5 (the paper's Table optimizations-
    performance compares its DFS and warp-centric forms the same way)."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    g = G.workload("chunglu1m")
    dg = gpm.graph_from_csr(g, stream=stream)
    out = {}
    for k in ((4, 5) if full else (4,)):
        c = gpm.gpm_clique_count(dg, k)
        wc = gpm.gpm_get_stats(dg)["kernel_ms"]
        cd = gpm.gpm_clique_count_dfs(dg, k)
        dfs = gpm.gpm_get_stats(dg)["kernel_ms"]
        out[f"k{k}"] = {"dm_dfs_kernel_ms": dfs, "warp_bitmap_kernel_ms": wc, "speedup": dfs / wc,
                        "same_counts": cd == c, "cliques": c}
    dg.close()
    return out


def listing_entry(stream) -> dict:
    """Subgraph listing (aggregate_store) through gpm_list: records per
    second delivered to a host consumer that counts them (motifs: by
    pattern, checked against gpm_motif_count), wall time of the whole call
    (the kernel writes into mapped host memory, the calling thread consumes
    while it runs)."""
    import torch
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    out = {}
    for name, app, k in (("rmat16", gpm.GPM_APP_CLIQUE, 4), ("rmat16", gpm.GPM_APP_CLIQUE, 5),
                         ("sbm2000", gpm.GPM_APP_CLIQUE, 6), ("er516", gpm.GPM_APP_MOTIF, 4),
                         ("sbm2000", gpm.GPM_APP_MOTIF, 4)):
        g = G.workload(name)
        dg = gpm.graph_from_csr(g, stream=stream)
        if app == gpm.GPM_APP_CLIQUE:
            want = np.array([gpm.gpm_clique_count(dg, k)], dtype=np.uint64)
        else:
            want = gpm.gpm_motif_count(dg, k)
        tally = np.zeros(want.shape[0], dtype=np.int64)

        def consume(recs):
            if app == gpm.GPM_APP_CLIQUE:
                tally[0] += recs.shape[0]
            else:
                tally[:] += np.bincount(recs[:, k], minlength=tally.shape[0])
            return False

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = gpm.gpm_list(dg, app, k, consume, ring_records=1 << 20)
        wall = time.perf_counter() - t0
        kern = gpm.gpm_get_stats(dg)["kernel_ms"]
        what = "clique" if app == gpm.GPM_APP_CLIQUE else "motif"
        out[f"{name}_{what}{k}"] = {"records": int(n), "wall_ms": wall * 1000.0, "kernel_ms": kern,
                                   "records_per_s": n / wall if wall > 0 else None,
                                   "ring_records": 1 << 20, "record_bytes": 4 * (k + 2),
                                   "same_as_counts": bool(np.array_equal(tally.astype(np.uint64), want))}
        dg.close()
    return out


def per_clique_entry(dg, g, k_lo, k_hi, counts, stream) -> dict:
    """The same step with the three-level tail's deepest level counted one
    AND + POPC per (k-1)-clique (clique_cpl = 0) instead of through the
    non-edges of dense nodes: same counts, the time it takes."""
    from paper_2212_04551_gb300 import gpm
    cfg = gpm.gpm_get_config(dg)
    gpm.gpm_set_config(dg, clique_cpl=0)
    try:
        c0, ms = timed(lambda: gpm.gpm_clique_count_range(dg, k_lo, k_hi), stream)
        st = gpm.gpm_get_stats(dg)
    finally:
        gpm.gpm_set_config(dg, cfg)
    total = sum(int(c) for c in c0)
    return {"clique_cpl": 0, "ms": ms, "kernel_ms": st["kernel_ms"], "subgraphs_per_s": total / (ms / 1000.0),
            "word_ops": int(st["word_ops"]), "same_counts": [int(x) for x in c0] == [int(x) for x in counts]}


def k4_8_entry(dg, g, stream) -> dict:
    """The configuration's full range: one enumeration to depth 8, timed
    once, and the 8-cliques of the stored 1/64 heaviest-first root sample
    checked root by root."""
    from paper_2212_04551_gb300 import gpm
    counts, ms = timed(lambda: gpm.gpm_clique_count_range(dg, 4, 8), stream)
    st = gpm.gpm_get_stats(dg)
    full = oracle_clique_totals(g)
    res = {"counts": {str(k): int(c) for k, c in zip(range(4, 9), counts)}, "ms": ms,
           "kernel_ms": st["kernel_ms"], "subgraphs_per_s": sum(int(c) for c in counts) / (ms / 1000.0),
           "word_ops": int(st["word_ops"]), "idle_warp_frac": st["idle_warp_frac"],
           "oracle_parity_full": {str(k): int(c) == full[k] for k, c in zip(range(4, 9), counts) if k in full}}
    gk = golden("chunglu1m_k78")
    if gk is not None and gk["sha256"] == g.sha256():
        sample = heaviest_first(g)[0::64]
        c8, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, 8, sample, per_root=True)
        want = np.zeros(g.n, dtype=np.uint64)
        for r, _, v8 in gk["k8_sample"]["per_root"]:
            want[r] = v8
        res["oracle_parity_k8_sample"] = {
            "roots": int(sample.shape[0]), "rule": gk["k8_sample"]["rule"],
            "total": int(c8[0]) == gk["k8_sample"]["cliques"]["8"],
            "per_root": bool(np.array_equal(pr, want[sample]))}
    return res


def _profile_case(name: str) -> None:
    """One launch of a kernel on a case small enough for an ncu capture
    (inputs larger than L2, a few hundred MB on the device, at most about a
    second), after one untimed launch of the same call."""
    import torch

    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    graph, run = PROFILE_CASES[name]
    g = G.workload(graph)
    dg = gpm.graph_from_csr(g, stream=stream)
    for _ in range(2):
        out = run(gpm, g, dg)
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "result": [int(x) for x in np.ravel(out)][:8], "stats": gpm.gpm_get_stats(dg)}))


PROFILE_CASES = {
    # the headline kernel: every root, k = 4..6 (two-level tail) and the
    # 1/64 heaviest-first sample at k = 7 (compacted three-level tail)
    "clique_chunglu1m_k4_6": ("chunglu1m", lambda gpm, g, dg: gpm.gpm_clique_count_range(dg, 4, 6)),
    # the headline step itself (one launch of about 5 s: capture only a few
    # sections of it)
    "clique_chunglu1m_k4_7": ("chunglu1m", lambda gpm, g, dg: gpm.gpm_clique_count_range(dg, 4, 7)),
    "clique_chunglu1m_k7_sample": ("chunglu1m", lambda gpm, g, dg: gpm.gpm_count_roots(
        dg, gpm.GPM_APP_CLIQUE, 7, heaviest_first(g)[0::64])[0]),
    # the bulk of the k = 7 search without its few heaviest roots (whose
    # split-up tails dominate a small sample): every 16th root from the
    # 1,024th heaviest on
    "clique_chunglu1m_k7_bulk": ("chunglu1m", lambda gpm, g, dg: gpm.gpm_count_roots(
        dg, gpm.GPM_APP_CLIQUE, 7, heaviest_first(g)[1024::16])[0]),
    # the motif kernel: marks in HBM (R-MAT, one heavy root) and in shared
    # memory (the block model graph)
    "motif_rmat16_k5_root132": ("rmat16", lambda gpm, g, dg: gpm.gpm_count_roots(
        dg, gpm.GPM_APP_MOTIF, 5, np.array([132], dtype=np.int32))[0]),
    "motif_sbm2000_k5": ("sbm2000", lambda gpm, g, dg: gpm.gpm_motif_count(dg, 5)),
}


def main():
    args = parse()
    if args.profile_case:
        _profile_case(args.profile_case)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2212_04551_gb300 import graphs as G

    kk = list(range(args.k_lo, args.k_hi + 1))
    config = {"workload": f"chunglu1m clique k={args.k_lo}..{args.k_hi}",
              "graph": "Chung-Lu n=1,000,000 avg deg 16 gamma 2.1 cap 20,000 seed 1, degree-ordered int32 CSR",
              "k": kk, "l2": "flushed between timed steps (512 MB write)",
              "parallelism": f"roots split over {world} rank(s)"}

    if args.impl == "reference":
        if rank != 0:
            return
        g = G.workload("chunglu1m")
        t_start = time.perf_counter()
        vals, descs, cores = [], [], 1
        for i in range(args.warmup + args.steps):
            v, desc, cores, _, _ = cpu_baseline(g, args.k_lo, args.k_hi, args.cpu_stride * 2, offset=1 + 2 * i)
            vals.append(v)
            descs.append(desc)
        v = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "ms_per_step": (time.perf_counter() - t_start) * 1000 / max(1, args.warmup + args.steps),
                "dtype": "int64", "data": "synthetic", "config": config, "vs_baseline": None,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": descs[-1] + "; one offset per step"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2212_04551_gb300 import gpm

    g = G.workload("chunglu1m")
    stream = torch.cuda.current_stream()
    ip = torch.from_numpy(g.indptr).cuda()
    ix = torch.from_numpy(g.indices).cuda()
    torch.cuda.synchronize()
    dg = gpm.gpm_graph_create(ip, ix, g.n, stream=stream)

    # this rank's roots: round-robin over the heaviest-first order
    outdeg = dag_out_degrees(g)
    order = np.argsort(-outdeg, kind="stable").astype(np.int32)
    order = order[outdeg[order] >= args.k_lo - 1]          # roots that can hold a k_lo-clique
    my_roots = order[rank::world] if world > 1 else None

    def step():
        if my_roots is None:
            return gpm.gpm_clique_count_range(dg, args.k_lo, args.k_hi)
        return [int(gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, my_roots)[0][0]) for k in kk]

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        counts = step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    step_ms, kern_ms, word_ops, idle_frac = [], [], [], []
    launches = 0
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        counts = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = gpm.gpm_get_stats(dg)
        kern_ms.append(st["kernel_ms"])
        word_ops.append(float(st["word_ops"]))
        idle_frac.append(st["idle_warp_frac"])
        launches += int(st["kernel_launches"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall_s = time.perf_counter() - t_wall
    clocks = sampler.stop()

    total = sum(int(c) for c in counts)
    t_step = statistics.mean(step_ms)
    if dist:
        tt = torch.tensor([t_step, float(total)], dtype=torch.float64, device="cuda")
        mx = tt.clone()
        dist.all_reduce(mx[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[1:], op=dist.ReduceOp.SUM)
        t_step, total = float(mx[0]), int(tt[1])
    value = total / (t_step / 1000.0)

    # end to end through the C ABI with host buffers
    h_ip, h_ix = g.indptr, g.indices
    e2e_ms = []
    for i in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hg = gpm.gpm_graph_create(h_ip, h_ix, g.n, stream=stream)
        if my_roots is None:
            c2 = gpm.gpm_clique_count_range(hg, args.k_lo, args.k_hi)
        else:
            c2 = [int(gpm.gpm_count_roots(hg, gpm.GPM_APP_CLIQUE, k, my_roots)[0][0]) for k in kk]
        hg.close()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1000)
        assert [int(x) for x in c2] == [int(x) for x in counts], "end-to-end counts differ"
    e2e_value = total / (statistics.mean(e2e_ms) / 1000.0)

    # roofline of the dominant kernel (k_clique), an integer-issue-bound
    # kernel: warp instructions issued per second against the SMs' issue
    # slots (4 schedulers x 1 instruction per clock per SM), with the
    # launch's instruction count from the committed ncu summary of the same
    # launch (identified by its exact word-operation count) and its time
    # measured here; beside it the word operations (AND + POPC of 32-bit
    # candidate words, counted exactly by the kernel) against the POPC rate
    hbm, sm_max, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    kern_s = statistics.mean(kern_ms) / 1000.0
    peak_ops = sms * POPC_PER_CLK_PER_SM * sm_max * 1e6
    peak_issue = sms * ISSUE_PER_CLK_PER_SM * sm_max * 1e6
    wops = statistics.mean(word_ops)
    src_hash = kernel_source_hash(["clique.cu", "clique_dev.cuh", "common.cuh"])
    prof = profiled_launch(f"k_clique_chunglu1m_k{args.k_lo}_{args.k_hi}.txt", src_hash, wops)
    word_line = {"achieved": wops / kern_s / 1e9, "peak": peak_ops / 1e9,
                 "unit": "Gop/s (32-bit candidate-word AND+POPC)", "frac": wops / kern_s / peak_ops,
                 "peak_kind": f"derived: {sms} SMs x {POPC_PER_CLK_PER_SM} POPC/clk x {sm_max:.0f} MHz",
                 "units_per_launch": wops}
    if prof:
        roofline = {"bound": "alu", "kernel": "k_clique", "achieved": prof["warp_inst"] / kern_s / 1e9,
                    "peak": peak_issue / 1e9, "unit": "G warp instructions/s",
                    "frac": prof["warp_inst"] / kern_s / peak_issue,
                    "peak_kind": f"derived: {sms} SMs x {ISSUE_PER_CLK_PER_SM} issue slots/clk x {sm_max:.0f} MHz "
                                 f"({peak_kind} clock)",
                    "units_per_launch": prof["warp_inst"], "traffic": prof["dram_bytes"],
                    "counts_from": f"profiles/k_clique_chunglu1m_k{args.k_lo}_{args.k_hi}.txt (ncu, same launch)",
                    "word_ops": word_line, "kernel_source_sha": src_hash}
    else:
        roofline = {"bound": "alu", "kernel": "k_clique", **word_line, "traffic": None,
                    "kernel_source_sha": src_hash}
    # HBM: DRAM bytes of the launch (ncu) over its time -- reported beside the
    # ALU roofline to show that memory bandwidth is not what binds the kernel
    traffic = roofline["traffic"]
    hbm_line = {"achieved_gbs": traffic / kern_s / 1e9 if traffic else None, "peak_gbs": hbm,
                "frac": traffic / kern_s / 1e9 / hbm if traffic else None,
                "peak_kind": f"{peak_kind} copy bandwidth", "bytes_per_launch": traffic}
    # parity at full size against the oracle's stored totals
    full = oracle_clique_totals(g)
    parity = None
    if world == 1 and all(k in full for k in kk):
        parity = {"oracle_full_size": all(int(c) == full[k] for k, c in zip(kk, counts)),
                  "source": "tests/golden/chunglu1m_full.json (k <= 6) and chunglu1m_k78.json (k = 7): "
                            "oracle over every root"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": config,
        "counts": {str(k): int(c) for k, c in zip(kk, counts)},
        "kernel_ms": statistics.mean(kern_ms), "wall_s": wall_s,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h_ip.nbytes + h_ix.nbytes),
                "d2h_bytes_per_step": 8 * len(kk), "ms_per_step": statistics.mean(e2e_ms)},
        "clocks": clocks, "gpu_launches": launches,
        "roofline": roofline, "hbm": hbm_line, "parity": parity,
        "sm_idle": {"idle_warp_frac": statistics.mean(idle_frac),
                    "definition": "1 - (sum over the grid's warps of time inside work units) / "
                                  "(warps x kernel time), %globaltimer"},
    }
    if rank == 0 and world == 1:
        line["deepest_level_per_clique"] = per_clique_entry(dg, g, args.k_lo, args.k_hi, counts, stream)
    if rank == 0 and world == 1 and not args.no_k8:
        line["k4_8"] = k4_8_entry(dg, g, stream)
    if rank == 0 and world == 1 and not args.no_configs:
        learned = Learned(stream)
        line["learned_training"] = learned.info
        line["configs"] = {"er516": config_er516(stream), "rmat16": config_rmat16(stream, learned, args.full),
                           "ba4096": config_ba4096(stream), "sbm2000": config_sbm2000(stream, learned)}
        line["ablations"] = {"balancing": balancing_ablation(stream, args.full),
                             "dm_dfs": dm_dfs_ablation(stream, args.full)}
        line["listing"] = listing_entry(stream)
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, cores, _, _ = cpu_baseline(g, args.k_lo, args.k_hi, args.cpu_stride)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
