"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts are integers, so the bar is bit-exact equality.  Motif counts are
compared per pattern: the library's pattern id p is mapped to its canonical
code with gpm_motif_pattern, and the oracle reports counts keyed by the same
canonical code (its own relabelling minimum).
"""
from __future__ import annotations

import functools
import json
import os
from math import comb

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpm.load()
    O.build()


def motif_by_code(g_dev, k) -> dict[int, int]:
    counts = gpm.gpm_motif_count(g_dev, k)
    return {gpm.gpm_motif_pattern(k, p): int(c) for p, c in enumerate(counts) if c}


def random_graph(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(2, 90))
    p = float(rng.uniform(0.02, 0.5))
    return G.gnp(n, p, seed)


# -------------------------------------------------------------- small graphs

@pytest.mark.parametrize("seed", range(40))
def test_clique_random_graphs(seed):
    g = random_graph(seed)
    dg = gpm.graph_from_csr(g)
    for k in range(1, 9):
        assert gpm.gpm_clique_count(dg, k) == O.clique_count(g, k), (seed, k)


@pytest.mark.parametrize("seed", range(40))
def test_motif_random_graphs(seed):
    g = random_graph(seed)
    dg = gpm.graph_from_csr(g)
    for k in range(1, 7):
        if comb(g.n, k) > 3_000_000:      # keep the oracle's share of the run short
            break
        assert motif_by_code(dg, k) == O.motif_count(g, k), (seed, k)


@pytest.mark.parametrize("agg_min", [0, 1, 16])
def test_motif_tail_modes(agg_min):
    """The last two motif levels counted leaf by leaf (agg_min 0) or by entry
    class (1: every node one level above the leaves; 16: nodes with at least
    16 entries left), on random graphs, a hub and planted blocks: the
    oracle's per-pattern counts, per root as well."""
    cases = [random_graph(s) for s in range(40, 52)] + [G.star(70), G.sbm(240, 40, 0.35, 0.03, 8),
                                                        G.disjoint_union(G.complete(9), G.path(6))]
    for g in cases:
        dg = gpm.graph_from_csr(g)
        gpm.gpm_set_config(dg, motif_agg_min=agg_min)
        for k in range(3, 7):
            if comb(g.n, k) > 3_000_000:
                break
            assert motif_by_code(dg, k) == O.motif_count(g, k), (g.n, k)
    g = G.gnp(60, 0.15, 41)
    dg = gpm.graph_from_csr(g)
    gpm.gpm_set_config(dg, motif_agg_min=agg_min, donate_after_us=0, donate_min=2)
    roots = np.arange(0, 60, 2, dtype=np.int32)
    for k in (4, 5, 6, 7):
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_MOTIF, k, roots, per_root=True)
        want, opr = O.motif_count(g, k, roots=roots, per_root=True)
        assert {gpm.gpm_motif_pattern(k, p): int(x) for p, x in enumerate(c) if x} == want, k
        assert np.array_equal(pr, opr), k


def test_motif_k7_random():
    for seed in range(4):
        g = G.gnp(40, 0.12, 900 + seed)
        dg = gpm.graph_from_csr(g)
        assert motif_by_code(dg, 7) == O.motif_count(g, 7)


def test_edge_cases():
    # empty graph, a single vertex, isolated vertices
    for g in (G.empty(0), G.empty(1), G.empty(17)):
        dg = gpm.graph_from_csr(g)
        assert gpm.gpm_clique_count(dg, 1) == g.n
        for k in (2, 3, 5):
            assert gpm.gpm_clique_count(dg, k) == 0
        assert int(gpm.gpm_motif_count(dg, 1)[0]) == g.n
        for k in (2, 3, 4):
            assert int(gpm.gpm_motif_count(dg, k).sum()) == 0
    # k above the largest clique; k = 2 gives m
    g = G.disjoint_union(G.complete(5), G.path(7), G.empty(3))
    dg = gpm.graph_from_csr(g)
    assert gpm.gpm_clique_count(dg, 6) == 0
    assert gpm.gpm_clique_count(dg, 2) == g.m
    assert gpm.gpm_clique_count(dg, 5) == 1


@pytest.mark.parametrize("n", [2, 33, 64, 65, 130, 300])
def test_complete_graphs(n):
    """K_n forces one full bitmap root of n-1 columns (multi-word rows)."""
    dg = gpm.graph_from_csr(G.complete(n))
    for k in (3, 4, 5):
        assert gpm.gpm_clique_count(dg, k) == comb(n, k)
    if n <= 65:
        for k in (6, 7):
            assert gpm.gpm_clique_count(dg, k) == comb(n, k)
    if n <= 64:
        got = gpm.gpm_motif_count(dg, 4)
        assert int(got.sum()) == comb(n, 4) and int(got[-1]) == comb(n, 4)


def test_turan_and_union():
    g = G.turan(60, 5)
    dg = gpm.graph_from_csr(g)
    parts = [12] * 5
    for k in range(1, 7):
        e = [1] + [0] * k
        for x in parts:
            for j in range(k, 0, -1):
                e[j] += e[j - 1] * x
        assert gpm.gpm_clique_count(dg, k) == e[k]


def _turan_cliques(parts, k):
    e = [1] + [0] * k
    for x in parts:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * x
    return e[k]


@functools.lru_cache(maxsize=1)
def _dense_reference():
    """Dense G(n, p) graphs (oriented out-degrees up to ~100: 3-4 words per
    bitmap row) with their oracle clique counts for k = 4, 5, 6."""
    out = []
    for seed, (n, p) in enumerate([(180, 0.5), (160, 0.6)]):
        g = G.gnp(n, p, 900 + seed)
        out.append((g, [O.clique_count(g, k) for k in (4, 5, 6)]))
    return out


@pytest.mark.parametrize("compact", [0, 1, 2])
def test_compacted_tail_dense_graphs(compact):
    """The two-level tail on the node's own members (clique_compact) against
    closed forms (K_n, Turan) and the oracle on dense random graphs whose
    oriented out-degrees need three to six words per bitmap row."""
    for n in (97, 150):
        dg = gpm.graph_from_csr(G.complete(n))
        gpm.gpm_set_config(dg, clique_compact=compact)
        assert [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 7)] == [comb(n, k) for k in range(4, 8)]
    dg = gpm.graph_from_csr(G.turan(200, 10))
    gpm.gpm_set_config(dg, clique_compact=compact, clique_tail=2)
    assert [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 7)] == [_turan_cliques([20] * 10, k)
                                                                     for k in range(4, 8)]
    for g, want in _dense_reference():
        dg = gpm.graph_from_csr(g)
        gpm.gpm_set_config(dg, clique_compact=compact)
        assert [gpm.gpm_clique_count(dg, k) for k in (4, 5, 6)] == want, g.n
        assert [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 6)] == want, g.n


@pytest.mark.parametrize("compact3", [0, 1, 2])
@pytest.mark.parametrize("cpl", [0, 1, 85])
def test_three_level_tail_modes(compact3, cpl):
    """The three-level clique tail (k >= 7) on the full-width rows (0), on
    the node's own members (1), and with the pairs of nodes of at most 64
    members taken by the whole warp (2); its deepest level counted per
    (k-1)-clique (cpl 0), through the non-edges of every node (1), or of
    nodes at least 85 % dense (85): closed forms on K_n and Turan graphs
    (member sets of 1 to 5 words; Turan parts give every node non-edges) and
    the oracle on dense random graphs and planted blocks."""
    for n, k_hi in ((40, 9), (70, 9), (97, 9), (150, 7)):
        dg = gpm.graph_from_csr(G.complete(n))
        gpm.gpm_set_config(dg, clique_compact3=compact3, clique_cpl=cpl)
        assert [int(x) for x in gpm.gpm_clique_count_range(dg, 4, k_hi)] == [comb(n, k) for k in range(4, k_hi + 1)], n
    for n, parts, k_hi in ((200, 10, 8), (96, 32, 9), (96, 48, 9)):
        dg = gpm.graph_from_csr(G.turan(n, parts))
        gpm.gpm_set_config(dg, clique_compact3=compact3, clique_cpl=cpl)
        assert [int(x) for x in gpm.gpm_clique_count_range(dg, 7, k_hi)] == [
            _turan_cliques([n // parts] * parts, k) for k in range(7, k_hi + 1)], (n, parts)
    for name, g, want in _dense_oracle_7_8():
        dg = gpm.graph_from_csr(g)
        gpm.gpm_set_config(dg, clique_compact3=compact3, clique_cpl=cpl, donate_after_us=0, donate_min=2)
        assert [int(x) for x in gpm.gpm_clique_count_range(dg, 7, 8)] == want, name
        assert [gpm.gpm_clique_count(dg, k) for k in (7, 8)] == want, name


@functools.lru_cache(maxsize=1)
def _dense_oracle_7_8():
    """Dense graphs with their oracle 7- and 8-clique counts (G(44, 0.9):
    nodes dense enough for the non-edge count; G(120, 0.55) and planted
    blocks: nodes that take the per-clique count under the default)."""
    out = []
    for name, g in (("gnp120", G.gnp(120, 0.55, 71)), ("gnp44", G.gnp(44, 0.9, 73)),
                    ("sbm500", G.sbm(500, 50, 0.6, 0.02, 72))):
        out.append((name, g, [O.clique_count(g, k) for k in (7, 8)]))
    return tuple(out)


def test_star_with_large_hub():
    """A hub of degree 300 (motifs) -- a long exclusive list in one step."""
    g = G.star(300)
    dg = gpm.graph_from_csr(g)
    for k in (2, 3, 4):
        got = gpm.gpm_motif_count(dg, k)
        assert int(got.sum()) == comb(300, k - 1)
    assert motif_by_code(dg, 4) == O.motif_count(g, 4)


def test_padding_boundaries():
    """Out-lists whose lengths straddle the 4-entry padding of the oriented CSR."""
    parts = [G.complete(s) for s in (3, 4, 5, 6, 7, 8, 9)]
    g = G.disjoint_union(*parts, G.path(11), G.cycle(13))
    dg = gpm.graph_from_csr(g)
    for k in range(3, 9):
        assert gpm.gpm_clique_count(dg, k) == O.clique_count(g, k)
    for k in (3, 4, 5):
        assert motif_by_code(dg, k) == O.motif_count(g, k)


def test_clique_range_matches_single():
    g = G.sbm(400, 50, 0.45, 0.02, 77)
    dg = gpm.graph_from_csr(g)
    rng_counts = gpm.gpm_clique_count_range(dg, 3, 9)
    for k in range(3, 10):
        assert rng_counts[k - 3] == O.clique_count(g, k)


# ---------------------------------------------------------- per-root parity

def test_per_root_clique_and_motif():
    g = G.gnp(70, 0.2, 123)
    dg = gpm.graph_from_csr(g)
    roots = np.arange(0, 70, 3, dtype=np.int32)
    for k in (3, 4, 5):
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, roots, per_root=True)
        tot, opr = O.clique_count(g, k, order=O.ORDER_DEGREE, roots=roots, per_root=True)
        assert int(c[0]) == tot and np.array_equal(pr, opr)
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_MOTIF, k, roots, per_root=True)
        want, opr = O.motif_count(g, k, roots=roots, per_root=True)
        got = {gpm.gpm_motif_pattern(k, p): int(x) for p, x in enumerate(c) if x}
        assert got == want and np.array_equal(pr, opr)


# -------------------------------------------------- scheduler independence

@functools.lru_cache(maxsize=1)
def _schedule_reference():
    g = G.sbm(600, 60, 0.4, 0.02, 5)
    return g, [O.clique_count(g, k) for k in (4, 6)], O.motif_count(g, 4)


@pytest.mark.parametrize("cfg", [
    dict(donate=0), dict(donate=1, donate_min=2, donate_after_us=0), dict(warps_per_block=4),
    dict(warps_per_block=16, blocks_per_sm=1), dict(order=gpm.GPM_ORDER_ID),
    dict(warps_per_block=1, blocks_per_sm=1), dict(clique_tail=2), dict(clique_tail=3, warps_per_block=2),
    dict(clique_compact=1), dict(clique_compact=2), dict(motif_agg_min=0), dict(motif_agg_min=1),
    dict(motif_agg_min=1, donate=1, donate_min=2, donate_after_us=0)])
def test_schedule_never_changes_counts(cfg):
    g, ref_c, ref_m = _schedule_reference()
    dg = gpm.graph_from_csr(g)
    gpm.gpm_set_config(dg, **cfg)
    assert [gpm.gpm_clique_count(dg, k) for k in (4, 6)] == ref_c
    assert motif_by_code(dg, 4) == ref_m


@pytest.mark.parametrize("threshold", [0.0, 0.4, 0.9])
def test_monitored_balancing_same_counts(threshold):
    """The paper's host-monitored stop / redistribute / restart balancing
    gives the in-kernel hand-off's counts, for cliques and motifs (and 5-
    and 7-cliques with the deeper tails)."""
    g, ref_c, ref_m = _schedule_reference()
    dg = gpm.graph_from_csr(g)
    c6, st = gpm.gpm_count_monitored(dg, gpm.GPM_APP_CLIQUE, 6, threshold)
    assert int(c6[0]) == ref_c[1]
    m4, st_m = gpm.gpm_count_monitored(dg, gpm.GPM_APP_MOTIF, 4, threshold)
    assert {gpm.gpm_motif_pattern(4, p): int(x) for p, x in enumerate(m4) if x} == ref_m
    for k in (5, 7):
        c, _ = gpm.gpm_count_monitored(dg, gpm.GPM_APP_CLIQUE, k, threshold)
        assert int(c[0]) == gpm.gpm_clique_count(dg, k), k
    m5, _ = gpm.gpm_count_monitored(dg, gpm.GPM_APP_MOTIF, 5, threshold)
    assert np.array_equal(m5, gpm.gpm_motif_count(dg, 5))
    if threshold == 0.0:
        assert st["launches"] == 1 and st["spilled_units"] == 0


def test_monitored_balancing_redistributes():
    """On the block-model workload (5-vertex motifs, 2,000 roots for a few
    thousand warps, ~0.2 s of work) the monitor at the paper's motif
    threshold stops the first launch while work is left, spills it and
    relaunches; the counts equal the oracle's."""
    g = G.workload("sbm2000")
    dg = gpm.graph_from_csr(g)
    m5, st = gpm.gpm_count_monitored(dg, gpm.GPM_APP_MOTIF, 5, 0.4)
    assert st["launches"] >= 2 and st["spilled_units"] > 0, st
    want = next(c["patterns"] for c in _golden("sbm2000_full")["cases"] if c["k"] == 5 and c["roots"] is None)
    assert {str(gpm.gpm_motif_pattern(5, p)): int(x) for p, x in enumerate(m5) if x} == want


# --------------------------------------------------------- invalid inputs

@pytest.mark.parametrize("bad", ["unsorted", "asymmetric", "selfloop", "duplicate", "range"])
def test_invalid_csr_rejected(bad):
    ip = np.array([0, 2, 4, 6], dtype=np.int32)
    ix = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)   # triangle
    if bad == "unsorted":
        ix = np.array([2, 1, 0, 2, 0, 1], dtype=np.int32)
    elif bad == "asymmetric":
        ix = np.array([1, 2, 0, 2, 1, 1], dtype=np.int32)
    elif bad == "selfloop":
        ix = np.array([0, 1, 0, 2, 0, 1], dtype=np.int32)
    elif bad == "duplicate":
        ix = np.array([1, 1, 0, 2, 0, 1], dtype=np.int32)
    elif bad == "range":
        ix = np.array([1, 7, 0, 2, 0, 1], dtype=np.int32)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_graph_create(ip, ix, 3)
    assert e.value.status == gpm.GPM_EINVAL
    gpm.gpm_graph_create(ip, ix, 3, flags=gpm.GPM_SKIP_VALIDATE).close()


def test_bounded_wait_times_out_and_recovers():
    """One heavy root whose warp never hands work over (donation on, but only
    after ~35 minutes of running): every other warp registers and waits on
    its mailbox while nothing completes, so with a 1 ms idle limit the wait
    runs out and the call returns GPM_ETIMEOUT (the busy warp sees the flag
    and stops); the same graph then counts correctly with the default
    limits."""
    g = G.complete(140)
    dg = gpm.graph_from_csr(g)
    root = np.array([0], dtype=np.int32)
    gpm.gpm_set_config(dg, donate=1, donate_after_us=2_000_000_000, max_idle_ms=1)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, 7, root)
    assert e.value.status == gpm.GPM_ETIMEOUT
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_count_roots(dg, gpm.GPM_APP_MOTIF, 6, root)
    assert e.value.status == gpm.GPM_ETIMEOUT
    gpm.gpm_set_config(dg, donate=1, donate_after_us=50, max_idle_ms=120000)
    assert gpm.gpm_clique_count(dg, 5) == comb(140, 5)
    got = gpm.gpm_motif_count(dg, 4)
    assert int(got.sum()) == comb(140, 4) and int(got[-1]) == comb(140, 4)


# ------------------------------------------------ stored workload values

def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{name}.json not generated")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["er516", "sbm2000", "rmat16", "chunglu1m", "rmat16_full", "sbm2000_full",
                                  "rmat16_strat"])
def test_workload_golden(name):
    """Full-size workloads, in the launch configuration the benchmark uses:
    full counts where the oracle finishes, else exact per-root counts on the
    seeded root samples stored beside them (the *_full files: every root, or
    the learned-scheduling comparison's 512 roots, by the oracle's ESU
    route; rmat16_strat: up to 16 roots per up-degree band at k = 5, 6, 7,
    the heaviest the oracle finishes within its per-root limit)."""
    data = _golden(name)
    g = G.workload(data["workload"])
    assert g.sha256() == data["sha256"]
    dg = gpm.graph_from_csr(g)
    for case in data["cases"]:
        k = case["k"]
        roots = case["roots"]
        if case["app"] == "clique":
            if roots is None:
                assert gpm.gpm_clique_count(dg, k) == case["total"], case["k"]
            else:
                c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, roots, per_root=True)
                assert int(c[0]) == case["total"]
                assert [int(x) for x in pr] == case["per_root"]
        else:
            want = {int(c): v for c, v in case["patterns"].items()}
            if roots is None:
                assert motif_by_code(dg, k) == want
            else:
                c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_MOTIF, k, roots, per_root=True)
                got = {gpm.gpm_motif_pattern(k, p): int(x) for p, x in enumerate(c) if x}
                assert got == want
                assert [int(x) for x in pr] == case["per_root"]


# ------------------------------------------ full-size properties (no oracle)

def _dominating(k, code):
    adj = [[False] * k for _ in range(k)]
    for i in range(1, k):
        for j in range(i):
            if (code >> (i * (i - 1) // 2 + j)) & 1:
                adj[i][j] = adj[j][i] = True
    return sum(1 for v in range(k) if all(adj[v][u] for u in range(k) if u != v))


def test_rmat16_full_size_identities():
    """R-MAT scale 16 (hub degree 6,444), whole graph: 3-motifs against the
    triangle count of the separate clique kernel and the wedge closed form
    sum C(d,2) - 3T; 4-motifs against the star identity
    sum_p dom(p) count_p = sum_v C(d(v), 3)."""
    g = G.workload("rmat16")
    dg = gpm.graph_from_csr(g)
    d = g.degrees()
    tri = gpm.gpm_clique_count(dg, 3)
    m3 = motif_by_code(dg, 3)
    codes3 = [gpm.gpm_motif_pattern(3, p) for p in range(2)]
    wedge_code, tri_code = codes3[0], codes3[1]
    assert bin(wedge_code).count("1") == 2 and tri_code == 7
    assert m3[tri_code] == tri
    assert m3[wedge_code] == sum(comb(int(x), 2) for x in d) - 3 * tri
    c4 = gpm.gpm_motif_count(dg, 4)
    lhs = sum(_dominating(4, gpm.gpm_motif_pattern(4, p)) * int(c) for p, c in enumerate(c4))
    assert lhs == sum(comb(int(x), 3) for x in d)


def test_rmat16_k5_every_root_star_identity():
    """5-vertex motifs over every root of R-MAT scale 16 -- the hub (degree
    6,444, id 0) roots about 7.6e13 of them -- in the benchmark's launch
    shape: sum_p dom(p) count_p = sum_v C(d(v), 4), with dom(p) the number of
    vertices of pattern p adjacent to all the others (every 5-set with a
    spanning star is connected, and is counted once per star centre); and
    the per-root totals add up to the pattern totals."""
    g = G.workload("rmat16")
    dg = gpm.graph_from_csr(g)
    d = g.degrees()
    c5, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_MOTIF, 5, None, per_root=True)
    lhs = sum(_dominating(5, gpm.gpm_motif_pattern(5, p)) * int(c) for p, c in enumerate(c5))
    assert lhs == sum(comb(int(x), 4) for x in d)
    assert sum(int(x) for x in pr) == sum(int(x) for x in c5)


def test_chunglu_full_counts_match_oracle():
    """The benchmark's workload and call at full size: one enumeration to
    depth 6 over every root of chunglu1m (gpm_clique_count_range) gives the
    4-, 5- and 6-clique totals the oracle computed over every root
    (tests/golden/chunglu1m_full.json, written by make_golden.py)."""
    with open(os.path.join(GOLDEN, "chunglu1m_full.json")) as f:
        data = json.load(f)
    g = G.workload("chunglu1m")
    assert g.sha256() == data["sha256"]
    dg = gpm.graph_from_csr(g)
    got = [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 6)]
    assert got == [data["cliques"][str(k)] for k in (4, 5, 6)]
    assert gpm.gpm_clique_count(dg, 3) == data["cliques"]["3"]


def test_chunglu_all_roots_per_root_matches_golden():
    """The benchmark's launch shape -- every root of chunglu1m in one launch,
    heaviest oriented out-degree first, donation on -- with per-root output:
    the counts of the 320 sampled roots equal the oracle's stored per-root
    values, and the per-root counts add up to the range call's totals."""
    data = _golden("chunglu1m")
    g = G.workload("chunglu1m")
    dg = gpm.graph_from_csr(g)
    d = g.degrees()
    e = g.edges()
    du, dv = d[e[:, 0]], d[e[:, 1]]
    fwd = (du < dv) | ((du == dv) & (e[:, 0] < e[:, 1]))
    outdeg = np.bincount(np.where(fwd, e[:, 0], e[:, 1]), minlength=g.n)
    order = np.argsort(-outdeg, kind="stable").astype(np.int32)
    pos = np.empty(g.n, dtype=np.int64)
    pos[order] = np.arange(g.n)
    totals = [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 6)]
    for k in (4, 5, 6):
        case = next(c for c in data["cases"] if c["app"] == "clique" and c["k"] == k)
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, order, per_root=True)
        assert int(c[0]) == totals[k - 4]
        assert sum(int(x) for x in pr) == totals[k - 4]
        assert [int(pr[pos[r]]) for r in case["roots"]] == case["per_root"], k


def test_chunglu_range_equals_single_counts():
    """Chung-Lu n = 1,000,000, the benchmark's launch: one DFS to depth 5
    gives the same 4- and 5-clique counts as two separate calls, and the
    triangle count matches the 3-motif triangle class of the motif kernel on
    a 20,000-vertex induced prefix (two independent kernels)."""
    g = G.workload("chunglu1m")
    dg = gpm.graph_from_csr(g)
    r = gpm.gpm_clique_count_range(dg, 4, 5)
    assert r == [gpm.gpm_clique_count(dg, 4), gpm.gpm_clique_count(dg, 5)]
    keep = 20000
    e = g.edges()
    e = e[(e[:, 0] < keep) & (e[:, 1] < keep)]
    h = G.from_edges(keep, e[:, 0], e[:, 1])
    dh = gpm.graph_from_csr(h)
    assert motif_by_code(dh, 3).get(7, 0) == gpm.gpm_clique_count(dh, 3)


# ------------------------------------------------------- overflow contract

@pytest.mark.parametrize("blocks,threads,where", [(1, 32, "lane"), (1, 32, "warp"), (1, 64, "block"),
                                                  (2, 32, "grid")])
def test_overflow_is_reported_not_wrapped(blocks, threads, where):
    """The kernels' reduction path (lane adds, warp sum, block counter,
    global counter) on values whose true sum is 2^64 (must return
    GPM_EOVERFLOW) and 2^64 - 1 (must return it exactly), with the two large
    values placed in one lane, two lanes of a warp, two warps of a block or
    two blocks."""
    nthreads = blocks * threads
    j = {"lane": nthreads, "warp": 1, "block": 32, "grid": 32}[where]
    v = np.zeros(2 * nthreads, dtype=np.uint64)
    v[0] = np.uint64(1 << 63)
    v[j] = np.uint64(1 << 63)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_selftest_sum(v, blocks, threads)
    assert e.value.status == gpm.GPM_EOVERFLOW
    v[j] = np.uint64((1 << 63) - 1)
    assert gpm.gpm_selftest_sum(v, blocks, threads) == (1 << 64) - 1


def test_selftest_sum_matches_python():
    """Many values over an odd launch shape: the exact sum when it fits
    (100,000 values below 2^40), GPM_EOVERFLOW when it does not (below
    2^50: the true sum is about 5.6e19 > 2^64)."""
    rng = np.random.default_rng(7)
    v = rng.integers(0, 1 << 40, size=100_000, dtype=np.uint64)
    assert gpm.gpm_selftest_sum(v, 37, 96) == int(v.astype(object).sum())
    w = rng.integers(0, 1 << 50, size=100_000, dtype=np.uint64)
    assert int(w.astype(object).sum()) >= 1 << 64
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_selftest_sum(w, 37, 96)
    assert e.value.status == gpm.GPM_EOVERFLOW


def _chunglu_heaviest_first(g):
    d = g.degrees()
    e = g.edges()
    du, dv = d[e[:, 0]], d[e[:, 1]]
    fwd = (du < dv) | ((du == dv) & (e[:, 0] < e[:, 1]))
    outdeg = np.bincount(np.where(fwd, e[:, 0], e[:, 1]), minlength=g.n)
    return np.argsort(-outdeg, kind="stable").astype(np.int32)


def test_chunglu_k7_every_root_matches_oracle():
    """The benchmark's launch shape at its deepest step size: every root of
    chunglu1m, heaviest oriented out-degree first, donation on, per-root
    output.  The 6- and 7-clique counts of every root (hashed, by vertex id)
    and their totals equal the oracle's bitset route over every root
    (tests/golden/chunglu1m_k78.json), and one enumeration to depth 7 gives
    the same totals."""
    import hashlib
    data = _golden("chunglu1m_k78")
    g = G.workload("chunglu1m")
    assert g.sha256() == data["sha256"]
    dg = gpm.graph_from_csr(g)
    order = _chunglu_heaviest_first(g)
    want = data["k7_all_roots"]
    for k in (6, 7):
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, order, per_root=True)
        assert int(c[0]) == want["cliques"][str(k)], k
        by_id = np.zeros(g.n, dtype="<u8")
        by_id[order] = pr
        assert hashlib.sha256(by_id.tobytes()).hexdigest() == want["per_root_sha256"][str(k)], k
    got = [int(x) for x in gpm.gpm_clique_count_range(dg, 4, 7)]
    assert got == [want["cliques"][str(k)] for k in (4, 5, 6, 7)]


def test_chunglu_k8_sample_per_root_matches_oracle():
    """8-cliques of the stored 1/64 sample of chunglu1m's roots (every 64th
    root of the heaviest-first order, starting at the heaviest), root by
    root, against the oracle's bitset route."""
    data = _golden("chunglu1m_k78")
    g = G.workload("chunglu1m")
    dg = gpm.graph_from_csr(g)
    sample = _chunglu_heaviest_first(g)[0::64]
    want = {r: (c7, c8) for r, c7, c8 in data["k8_sample"]["per_root"]}
    c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, 8, sample, per_root=True)
    assert int(c[0]) == data["k8_sample"]["cliques"]["8"]
    assert [int(x) for x in pr] == [want.get(int(r), (0, 0))[1] for r in sample]
    c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, 7, sample, per_root=True)
    assert int(c[0]) == data["k8_sample"]["cliques"]["7"]
    assert [int(x) for x in pr] == [want.get(int(r), (0, 0))[0] for r in sample]


# ------------------------------------------------------- 8-vertex motifs

def test_motif_k8():
    """8-vertex motifs (11,117 patterns; counted leaf by leaf into global
    pattern counters): the oracle's ESU route per pattern on two random
    graphs, closed forms on a path and a star, and the star identity
    sum_p dom(p) count_p = sum_v C(d(v), 7) on a sparse random graph."""
    for g in (G.gnp(40, 0.1, 2), G.gnp(28, 0.16, 5)):
        dg = gpm.graph_from_csr(g)
        assert motif_by_code(dg, 8) == O.motif_count(g, 8, method="esu")
    dg = gpm.graph_from_csr(G.path(20))
    assert list(motif_by_code(dg, 8).values()) == [13]
    dg = gpm.graph_from_csr(G.star(12))
    assert list(motif_by_code(dg, 8).values()) == [comb(12, 7)]
    g = G.gnp(400, 0.012, 9)
    dg = gpm.graph_from_csr(g)
    c8 = gpm.gpm_motif_count(dg, 8)
    lhs = sum(_dominating(8, gpm.gpm_motif_pattern(8, p)) * int(c) for p, c in enumerate(c8) if c)
    assert lhs == sum(comb(int(x), 7) for x in g.degrees())
    assert int(c8.sum()) > 0


def test_dm_dfs_baseline_counts():
    """The paper's DM_DFS baseline kernel (one thread per root, merged
    sorted lists) against closed forms and the oracle."""
    for n in (2, 9, 40):
        dg = gpm.graph_from_csr(G.complete(n))
        assert [gpm.gpm_clique_count_dfs(dg, k) for k in range(2, 7)] == [comb(n, k) for k in range(2, 7)]
    for g in (G.gnp(120, 0.3, 81), G.sbm(500, 50, 0.5, 0.02, 82), G.turan(60, 6)):
        dg = gpm.graph_from_csr(g)
        for k in (3, 4, 5, 6):
            assert gpm.gpm_clique_count_dfs(dg, k) == O.clique_count(g, k), (g.n, k)
