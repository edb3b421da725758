"""The batched persistent launch: per-graph counts from one captured launch
equal the oracle's per graph; replays, autotuned shapes and unit orders give
identical counts."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_batch():
    rng = np.random.default_rng(42)
    gs = G.barabasi_albert_batch(60, 8, 90, 2, 6, seed=17)
    gs += [G.gnp(int(rng.integers(2, 40)), float(rng.uniform(0.05, 0.5)), 1000 + i) for i in range(20)]
    gs += [G.empty(0), G.empty(5), G.complete(12), G.star(30), G.path(9)]
    return gs


def _expected(gs, kc, km):
    cc = [O.clique_count(g, kc) for g in gs]
    mc = [O.motif_count(g, km) for g in gs]
    return cc, mc


def _to_codes(row, km):
    return {gpm.gpm_motif_pattern(km, p): int(x) for p, x in enumerate(row) if x}


@pytest.mark.parametrize("kc,km", [(4, 5), (3, 4), (5, 3)])
def test_batch_matches_oracle(small_batch, kc, km):
    b = gpm.batch_from_graphs(small_batch)
    cc, mc = gpm.gpm_batch_count(b, kc, km)
    want_c, want_m = _expected(small_batch, kc, km)
    assert [int(x) for x in cc] == want_c
    for i, row in enumerate(mc):
        assert _to_codes(row, km) == want_m[i], i
    # replay of the captured graph gives the same numbers
    cc2, mc2 = gpm.gpm_batch_count(b, kc, km)
    assert np.array_equal(cc, cc2) and np.array_equal(mc, mc2)


def test_batch_single_task_and_shapes(small_batch):
    b = gpm.batch_from_graphs(small_batch)
    ref_c, ref_m = gpm.gpm_batch_count(b, 4, 5)
    cc, none = gpm.gpm_batch_count(b, 4, 0)
    assert none is None and np.array_equal(cc, ref_c)
    none, mc = gpm.gpm_batch_count(b, 0, 5)
    assert none is None and np.array_equal(mc, ref_m)
    for wpb, bps in [(2, 0), (4, 1), (16, 2), (1, 0)]:
        gpm.gpm_batch_set_config(b, warps_per_block=wpb, blocks_per_sm=bps)
        cc, mc = gpm.gpm_batch_count(b, 4, 5)
        assert np.array_equal(cc, ref_c) and np.array_equal(mc, ref_m), (wpb, bps)
    # the other tuned knobs: class-counting threshold and heavy-root split
    for agg, split in [(0, 1), (1, 1), (4, 16), (64, 4), (16, 64)]:
        gpm.gpm_batch_set_config(b, warps_per_block=4, motif_agg_min=agg, batch_split=split)
        cc, mc = gpm.gpm_batch_count(b, 4, 5)
        assert np.array_equal(cc, ref_c) and np.array_equal(mc, ref_m), (agg, split)
    best, ms = gpm.gpm_batch_autotune(b, 4, 5, reps=1)
    assert best["warps_per_block"] in (2, 4, 8, 16)
    assert best["motif_agg_min"] in (0, 4, 16, 64) and best["batch_split"] in (1, 4, 16)
    cc, mc = gpm.gpm_batch_count(b, 4, 5)
    assert np.array_equal(cc, ref_c) and np.array_equal(mc, ref_m)


def test_batch_matches_single_graph_calls():
    gs = G.barabasi_albert_batch(200, 20, 400, 2, 6, seed=3)
    b = gpm.batch_from_graphs(gs)
    cc, mc = gpm.gpm_batch_count(b, 4, 5)
    for i in range(0, 200, 23):
        dg = gpm.graph_from_csr(gs[i])
        assert int(cc[i]) == gpm.gpm_clique_count(dg, 4)
        assert np.array_equal(mc[i], gpm.gpm_motif_count(dg, 5))
    # sampled graphs against the oracle
    for i in (0, 57, 199):
        assert int(cc[i]) == O.clique_count(gs[i], 4)
        assert _to_codes(mc[i], 5) == O.motif_count(gs[i], 5)


def test_batch_rejects_cross_graph_edges():
    goff = np.array([0, 2, 4], dtype=np.int32)
    indptr = np.array([0, 1, 3, 4, 5], dtype=np.int32)
    indices = np.array([1, 0, 2, 1, 2], dtype=np.int32)   # edge 1-2 crosses graphs (and 3's list is bad)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_batch_create(goff, indptr, indices)
    assert e.value.status == gpm.GPM_EINVAL


def test_ba4096_golden():
    """The full 4,096-graph Barabasi-Albert batch in the benchmark's launch
    configuration (autotuned shape, CUDA-graph replay): per-graph 4-clique and
    5-motif counts of 48 seeded graphs equal the oracle's stored values
    (tests/golden/ba4096.json, written by make_golden.py from oracle/ only),
    and every graph satisfies the star identity of its 5-motif counts."""
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ba4096.json")) as f:
        data = json.load(f)
    gs = list(G.workload("ba4096"))
    import hashlib
    h = hashlib.sha256()
    for g in gs:
        h.update(g.sha256().encode())
    assert h.hexdigest() == data["sha256"]
    b = gpm.batch_from_graphs(gs)
    gpm.gpm_batch_autotune(b, 4, 5, reps=1)
    cc, mc = gpm.gpm_batch_count(b, 4, 5)
    for i, c4, m5 in zip(data["graphs"], data["clique4"], data["motif5"]):
        assert int(cc[i]) == c4, i
        assert _to_codes(mc[i], 5) == {int(c): v for c, v in m5.items()}, i
    # every graph, at full size: the star identity sum_p dom(p) count_p =
    # sum_v C(d(v), 4) (each connected 5-set with a vertex adjacent to all
    # others is counted once per such vertex)
    from math import comb
    dom = []
    for pid in range(mc.shape[1]):
        code = gpm.gpm_motif_pattern(5, pid)
        adj = [[False] * 5 for _ in range(5)]
        for a in range(1, 5):
            for c in range(a):
                if (code >> (a * (a - 1) // 2 + c)) & 1:
                    adj[a][c] = adj[c][a] = True
        dom.append(sum(1 for v in range(5) if all(adj[v][u] for u in range(5) if u != v)))
    for i, g in enumerate(gs):
        lhs = sum(int(x) * d for x, d in zip(mc[i], dom))
        assert lhs == sum(comb(int(d), 4) for d in g.degrees()), i
    # replaying the captured launch gives the same numbers
    cc2, mc2 = gpm.gpm_batch_count(b, 4, 5)
    assert np.array_equal(cc, cc2) and np.array_equal(mc, mc2)
