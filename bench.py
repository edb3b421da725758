"""Benchmark: enumerated subgraphs/s on one GB300 (bit-exact counts).

Default workload (the plain method at scale): k-clique counting on the
Chung-Lu power-law graph (n = 1,000,000, average degree 16, exponent 2.1,
expected degrees capped at 20,000, seed 1), degree-ordered, int32 CSR.  One
step = one enumeration that counts every clique size k_lo..k_hi
(gpm_clique_count_range), with the graph already resident in HBM.  The
default range is 4..6 (a step of about half a second); ``--k-hi 7`` and
``--k-hi 8`` run deeper ranges of the same configuration (seconds to hours:
the 8-clique count is about 1e15).

Printed: one JSON line (rank 0) with the metric, the device-timed value,
the end-to-end value through the C ABI with host buffers (graph creation
from host CSR + counting + result read-back inside the timed region), the
roofline of the dominant kernel, SM clocks sampled during the timed region,
and the CPU oracle timed on a bounded root sample of the same workload.

``--impl reference`` times the CPU oracle alone on that bounded sample (the
reference arm for this method is the plain CPU restatement of the paper's
enumeration).

Multi-GPU (torchrun, N ranks): the roots are split round-robin over the
ranks -- every clique has exactly one root -- and the per-rank counts are
summed on the host; value = all subgraphs / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

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
    ap.add_argument("--k-hi", type=int, default=6)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the learned and batched comparisons")
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


def kernel_source_hash(names) -> str:
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2212_04551_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary: str, src_hash: str, units_now: float):
    """DRAM bytes per launch from a committed ncu summary of the same launch,
    or None when the kernel source changed since or the launch differs (the
    clique kernel's DRAM bytes are the per-root row builds, which do not grow
    with the word operations of deeper k ranges, so they are not scaled)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != src_hash:
        return None
    try:
        t = float(kv["dram_bytes_per_launch"])
        u = float(kv["units_per_launch"])
    except (KeyError, ValueError):
        return None
    return t if u > 0 and abs(units_now - u) <= 1e-6 * u else None


def golden(name: str):
    """A stored oracle result under tests/golden/ (written by make_golden.py
    from the oracle only), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def oracle_full_size(k_lo: int, k_hi: int):
    """Full-size clique counts of chunglu1m and the list-merge bytes of the
    depth-6 search, computed by the oracle over every root and stored by
    tests/golden/make_golden.py (None when absent or not covering k_hi)."""
    path = os.path.join(ROOT, "tests", "golden", "chunglu1m_full.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return d if k_hi <= d["k_max"] else None


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


def cpu_baseline(g, k_lo, k_hi, budget_s):
    """The oracle, as it stands, on a bounded seeded root sample of the same
    workload: roots drawn uniformly, counted one k at a time until the time
    budget is spent.  Returns (subgraphs/s, description, roots used)."""
    from oracle import oracle as O
    from paper_2212_04551_gb300 import graphs as G
    O.build()
    perm = G.sample_roots(g.n, g.n, seed=99)          # all roots, seeded order
    rng = np.random.default_rng(99)
    rng.shuffle(perm)
    done = 0
    found = 0
    t0 = time.perf_counter()
    chunk = 64
    while time.perf_counter() - t0 < budget_s and done < g.n:
        roots = perm[done:done + chunk]
        for k in range(k_lo, k_hi + 1):
            found += O.clique_count(g, k, order=O.ORDER_DEGREE, roots=roots)
        done += roots.shape[0]
    el = time.perf_counter() - t0
    desc = (f"oracle clique k={k_lo}..{k_hi} (Algorithm 4, one k per pass) on {done} seeded uniform roots "
            f"of {g.n} ({el:.1f} s, single thread)")
    return found / el, desc, done


def timed(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def learned_vs_plain(stream, k: int = 5, n_roots: int = 512, epochs: int = 60, reps: int = 2) -> dict:
    """Learned scheduling (the MLP trained on R-MAT scale-12 graphs, seeds
    100-131, with per-root sizes measured by the plain enumerator) against the
    plain heaviest-degree-first donation scheduler, on the R-MAT scale-16 graph
    restricted to a seeded sample of roots (ids >= 1024, degree <= 32);
    counts must agree exactly."""
    import torch

    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    from paper_2212_04551_gb300 import learned as L
    t0 = time.perf_counter()
    X, T = L.training_set(gpm.GPM_APP_MOTIF, k, seeds=range(100, 132), scale=12, stream=stream)
    t_labels = time.perf_counter() - t0
    model = L.new_model(0, stream)
    untrained = L.new_model(0, stream)
    t0 = time.perf_counter()
    L.train(model, X, T, epochs=epochs, batch=4096, lr=3e-3, stream=stream)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    g = G.workload("rmat16")
    d = g.degrees()
    ok = (np.arange(g.n) >= 1024) & (d <= 32)
    roots = G.sample_roots(g.n, n_roots, seed=25, exclude=~ok)
    dg = gpm.graph_from_csr(g, stream=stream)
    feats = L.features(dg, g.n)
    pred_trained = L.predict(model, feats, stream)
    pred_untrained = L.predict(untrained, feats, stream)
    res = {}
    ref = None
    sizes = None
    for donate in (1, 0):
        gpm.gpm_set_config(dg, donate=donate)
        tag = "donation" if donate else "static"
        res[tag] = {}
        for name, pred in (("plain", None), ("learned", pred_trained), ("untrained", pred_untrained)):
            if pred is None:
                gpm.gpm_sched_from_scores(dg, gpm.GPM_APP_MOTIF, None, roots, 0, 0)
                plan = {"split_roots": 0, "chunks": 0}
            else:
                plan = L.schedule(dg, gpm.GPM_APP_MOTIF, pred, roots, warps=4864, chunks=8)
            times = []
            for _ in range(reps):
                (c, pr), ms = timed(lambda: gpm.gpm_count_scheduled(dg, gpm.GPM_APP_MOTIF, k, n_roots=len(roots),
                                                                    per_root=True), stream)
                times.append(ms)
            st = gpm.gpm_get_stats(dg)
            if ref is None:
                ref, sizes = c, pr
            assert np.array_equal(c, ref), f"{name} schedule changed the counts"
            ms = statistics.median(times)
            res[tag][name] = {"ms": ms, "subgraphs_per_s": int(ref.sum()) / (ms / 1000.0),
                              "donations": int(st["donations"]), "units": int(st["units_done"]),
                              "idle_warp_frac": st["idle_warp_frac"], **plan}
        res[tag]["speedup_learned_vs_plain"] = res[tag]["plain"]["ms"] / res[tag]["learned"]["ms"]
    from scipy.stats import spearmanr
    meas = np.log1p(sizes.astype(np.float64))
    res["spearman_trained"] = float(spearmanr(pred_trained.cpu().numpy()[roots], meas).statistic)
    res["spearman_untrained"] = float(spearmanr(pred_untrained.cpu().numpy()[roots], meas).statistic)
    res["spearman_degree"] = float(spearmanr(g.degrees()[roots], meas).statistic)
    res["k"] = k
    res["roots"] = f"{len(roots)} seeded roots of rmat16 (id >= 1024, degree <= 32)"
    gd = golden("rmat16_full")
    case = None if gd is None else next((c for c in gd["cases"] if c["k"] == k and c["roots"] is not None), None)
    if case is not None and case["roots"] == [int(r) for r in roots]:
        got = {str(gpm.gpm_motif_pattern(k, p)): int(x) for p, x in enumerate(ref) if x}
        res["oracle_parity"] = got == case["patterns"] and [int(x) for x in sizes] == case["per_root"]
    res["subgraphs"] = int(ref.sum())
    res["train"] = {"samples": int(X.shape[0]), "epochs": epochs, "label_s": round(t_labels, 2),
                    "train_s": round(t_train, 2), "final_mse": model.history[-1], "first_mse": model.history[0]}
    dg.close()
    return res


def batched_vs_plain(stream, reps: int = 5) -> dict:
    """4,096 Barabasi-Albert graphs, per-graph 4-clique and 5-motif counts:
    one autotuned, CUDA-graph-captured persistent launch against the plain
    form (one gpm_clique_count + one gpm_motif_count per graph)."""
    from paper_2212_04551_gb300 import gpm
    from paper_2212_04551_gb300 import graphs as G
    gs = list(G.workload("ba4096"))
    b = gpm.batch_from_graphs(gs, stream=stream)
    best, _ = gpm.gpm_batch_autotune(b, 4, 5, reps=3)
    cc, mc = gpm.gpm_batch_count(b, 4, 5)
    times = []
    for _ in range(reps):
        _, ms = timed(lambda: gpm.gpm_batch_count(b, 4, 5), stream)
        times.append(ms)
    total = int(cc.sum()) + int(mc.sum())
    parity = None
    gd = golden("ba4096")
    if gd is not None:
        parity = all(int(cc[i]) == c4 and {str(gpm.gpm_motif_pattern(5, p)): int(x)
                                           for p, x in enumerate(mc[i]) if x} == m5
                     for i, c4, m5 in zip(gd["graphs"], gd["clique4"], gd["motif5"]))
    t_b = statistics.median(times)
    idle_b = gpm.gpm_batch_get_stats(b)["idle_warp_frac"]
    # plain: every graph on its own, graphs resident on the device
    dgs = [gpm.graph_from_csr(g, stream=stream) for g in gs]
    def plain():
        c = np.array([gpm.gpm_clique_count(d, 4) for d in dgs], dtype=np.uint64)
        m = np.stack([gpm.gpm_motif_count(d, 5) for d in dgs])
        return c, m
    (pc, pm), t_p = timed(plain, stream)
    assert np.array_equal(pc, cc) and np.array_equal(pm, mc), "batched counts differ from per-graph counts"
    for d in dgs:
        d.close()
    b.close()
    return {"graphs": len(gs), "subgraphs": total, "batched_ms": t_b, "plain_ms": t_p,
            "batched_subgraphs_per_s": total / (t_b / 1000.0), "plain_subgraphs_per_s": total / (t_p / 1000.0),
            "speedup": t_p / t_b, "autotuned": best, "batched_idle_warp_frac": idle_b,
            "oracle_parity_48_graphs": parity}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2212_04551_gb300 import graphs as G

    config = {"workload": f"chunglu1m clique k={args.k_lo}..{args.k_hi}",
              "graph": "Chung-Lu n=1,000,000 avg deg 16 gamma 2.1 cap 20,000 seed 1, degree-ordered int32 CSR",
              "k": list(range(args.k_lo, args.k_hi + 1)),
              "l2": "flushed between timed steps (512 MB write)", "parallelism": f"roots split over {world} rank(s)"}

    if args.impl == "reference":
        if rank != 0:
            return
        g = G.workload("chunglu1m")
        t_start = time.perf_counter()
        vals = []
        for _ in range(args.warmup + args.steps):
            v, desc, _ = cpu_baseline(g, args.k_lo, args.k_hi, args.cpu_seconds / max(1, args.steps))
            vals.append(v)
        v = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "ms_per_step": (time.perf_counter() - t_start) * 1000 / max(1, args.warmup + args.steps),
                "dtype": "int64", "data": "synthetic", "config": config, "vs_baseline": None,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
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
    kk = list(range(args.k_lo, args.k_hi + 1))

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

    # roofline of the dominant kernel (k_clique): ALU-bound on population
    # counts of candidate words; achieved = word operations per launch (the
    # kernel counts them exactly) / the launch's CUDA-event time
    hbm, sm_max, peak_kind = peaks()
    import torch as _t
    sms = _t.cuda.get_device_properties(local_rank).multi_processor_count
    peak_ops = sms * POPC_PER_CLK_PER_SM * sm_max * 1e6
    wops = statistics.mean(word_ops)
    achieved = wops / (statistics.mean(kern_ms) / 1000.0)
    src_hash = kernel_source_hash(["clique.cu", "clique_dev.cuh", "common.cuh"])
    roofline = {"bound": "alu", "kernel": "k_clique", "achieved": achieved / 1e9, "peak": peak_ops / 1e9,
                "unit": "Gop/s (32-bit candidate-word AND+POPC)", "frac": achieved / peak_ops,
                "peak_kind": f"derived: {sms} SMs x {POPC_PER_CLK_PER_SM} POPC/clk x {sm_max:.0f} MHz ({peak_kind} clock)",
                "units_per_launch": wops,
                "traffic": profiled_traffic("k_clique_chunglu1m.txt", src_hash, wops),
                "kernel_source_sha": src_hash}
    # HBM: DRAM bytes of the launch (ncu) over its time -- reported beside the
    # ALU roofline to show that memory bandwidth is not what binds the kernel
    kern_s = statistics.mean(kern_ms) / 1000.0
    traffic = roofline["traffic"]
    hbm_line = {"achieved_gbs": traffic / kern_s / 1e9 if traffic else None, "peak_gbs": hbm,
                "frac": traffic / kern_s / 1e9 / hbm if traffic else None,
                "peak_kind": f"{peak_kind} copy bandwidth", "bytes_per_launch": traffic}
    # parity at full size against the oracle's stored totals, and the bytes a
    # sorted-list merge enumerator would move for the same search (B_alg),
    # expressed against the measured HBM bandwidth
    full = oracle_full_size(args.k_lo, args.k_hi)
    parity = None
    list_merge = None
    if full is not None and world == 1 and full["sha256"] == g.sha256():
        parity = {"oracle_full_size": all(int(c) == full["cliques"][str(k)] for k, c in zip(kk, counts)),
                  "source": "tests/golden/chunglu1m_full.json (oracle over every root)"}
        if args.k_hi == full["k_max"]:
            b = float(full["b_alg_depth6"])
            list_merge = {"b_alg_bytes_per_step": b, "gbs": b / (t_step / 1000.0) / 1e9,
                          "x_measured_hbm_peak": b / (t_step / 1000.0) / 1e9 / hbm,
                          "definition": "sum over node expansions of 4 (|C(S)| + d+(v)) bytes (sorted-list merge)"}
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
        "roofline": roofline, "hbm": hbm_line, "parity": parity, "list_merge_equivalent": list_merge,
        "sm_idle": {"idle_warp_frac": statistics.mean(idle_frac),
                    "definition": "1 - (sum over the grid's warps of time inside work units) / "
                                  "(warps x kernel time), %globaltimer"},
    }
    if rank == 0 and world == 1 and not args.no_variants:
        line["batched_vs_plain"] = batched_vs_plain(stream)
        line["learned_vs_plain"] = learned_vs_plain(stream)
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, _ = cpu_baseline(g, args.k_lo, args.k_hi, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
