"""Subgraph listing with an asynchronous host consumer (aggregate_store):
gpm_list through the C ABI.

What is checked, with nothing taken from the CUDA path as expected values:

* every record is a valid subgraph (its vertices pairwise adjacent for a
  clique; connected for a motif), records are distinct as vertex sets, and
  there are exactly as many as the CPU oracle counts -- so the listed sets
  are exactly the counted ones;
* for small graphs, the clique sets equal networkx's clique enumeration;
* each motif record's pattern id names the canonical code the oracle
  computes for the record's induced subgraph, and per pattern the records
  number what the oracle counts;
* the query form (one pattern id) lists that pattern's subgraphs only;
* rings far smaller than the output (records wrap around many times and the
  device waits for the consumer), a consumer that stops early, a consumer
  that is too slow (the device's bounded wait runs out: GPM_ETIMEOUT, and
  the graph stays usable), and bad arguments.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpm.load()
    O.build()


class Collect:
    """Consumer that keeps copies of every batch."""

    def __init__(self, stop_after=None, sleep_first=0.0):
        self.parts = []
        self.calls = 0
        self.stop_after = stop_after
        self.sleep_first = sleep_first

    def __call__(self, recs):
        self.calls += 1
        if self.calls == 1 and self.sleep_first:
            time.sleep(self.sleep_first)
        self.parts.append(np.array(recs, copy=True))
        return self.stop_after is not None and self.calls >= self.stop_after

    def records(self, k):
        if not self.parts:
            return np.zeros((0, k + 1), dtype=np.int32)
        return np.concatenate(self.parts)


def _adj_matrix(g):
    A = np.zeros((g.n, g.n), dtype=bool)
    e = g.edges()
    A[e[:, 0], e[:, 1]] = True
    A[e[:, 1], e[:, 0]] = True
    return A


def _distinct_sets(ids):
    s = np.sort(ids, axis=1)
    return np.unique(s, axis=0).shape[0] == s.shape[0]


def _check_cliques(g, k, recs, A=None):
    ids = recs[:, :k]
    assert (recs[:, k] == -1).all()
    assert ids.min() >= 0 and ids.max() < g.n
    A = _adj_matrix(g) if A is None else A
    for i in range(k):
        for j in range(i + 1, k):
            assert A[ids[:, i], ids[:, j]].all()
    assert _distinct_sets(ids)


def _induced_codes(A, ids, k):
    code = np.zeros(ids.shape[0], dtype=np.uint64)
    for i in range(1, k):
        for j in range(i):
            bit = np.uint64(1) << np.uint64(i * (i - 1) // 2 + j)
            code |= np.where(A[ids[:, j], ids[:, i]], bit, np.uint64(0))
    return code


def _check_motifs(g, k, recs, A=None):
    """Records are distinct connected k-sets whose pattern ids match the
    oracle's canonical codes; returns the per-code record counts."""
    A = _adj_matrix(g) if A is None else A
    ids = recs[:, :k]
    assert ids.min() >= 0 and ids.max() < g.n
    assert _distinct_sets(ids)
    codes, inv = np.unique(_induced_codes(A, ids, k), return_inverse=True)
    canon = O.canon_many(k, codes)[inv.ravel()]
    pat = {p: gpm.gpm_motif_pattern(k, p) for p in np.unique(recs[:, k])}
    want = np.array([pat[p] for p in recs[:, k]], dtype=np.uint64)
    assert np.array_equal(canon, want)
    assert all(O.code_connected(k, int(c)) for c in np.unique(canon))
    u, cnt = np.unique(canon, return_counts=True)
    return {int(a): int(b) for a, b in zip(u, cnt)}


@pytest.mark.parametrize("seed", range(6))
def test_clique_listing_matches_networkx(seed):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(300 + seed)
    g = G.gnp(int(rng.integers(20, 70)), float(rng.uniform(0.2, 0.6)), 310 + seed)
    h = nx.Graph()
    h.add_nodes_from(range(g.n))
    h.add_edges_from(map(tuple, g.edges()))
    by_size = {}
    for c in nx.enumerate_all_cliques(h):
        by_size.setdefault(len(c), set()).add(tuple(sorted(c)))
    dg = gpm.graph_from_csr(g)
    for k in (3, 4, 5, 6):
        col = Collect()
        n = gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, k, col, ring_records=64 + 32 * seed)
        recs = col.records(k)
        assert n == recs.shape[0] == len(by_size.get(k, ()))
        got = {tuple(sorted(int(x) for x in r[:k])) for r in recs}
        assert got == by_size.get(k, set())
        if n:
            _check_cliques(g, k, recs)


def test_clique_listing_wraps_a_small_ring():
    """About 130,000 4-cliques through a 64-record ring (thousands of
    wrap-arounds, the device waiting on the consumer)."""
    g = G.sbm(600, 60, 0.55, 0.01, 5)
    k = 4
    want = O.clique_count(g, k)
    assert want > 100_000
    dg = gpm.graph_from_csr(g)
    for ring in (64, 100_003):
        col = Collect()
        n = gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, k, col, ring_records=ring)
        recs = col.records(k)
        assert n == recs.shape[0] == want
        _check_cliques(g, k, recs)


@pytest.mark.parametrize("k", [3, 4, 5, 6, 8])
def test_motif_listing_matches_oracle(k):
    g = G.gnp(20, 0.15, 708) if k == 8 else G.gnp(60, 0.08, 700 + k)
    dg = gpm.graph_from_csr(g)
    want = O.motif_count(g, k)
    col = Collect()
    n = gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, k, col, ring_records=256)
    recs = col.records(k)
    assert n == recs.shape[0] == sum(want.values())
    assert _check_motifs(g, k, recs) == want
    # the counting path agrees pattern by pattern
    counts = gpm.gpm_motif_count(dg, k)
    got = np.bincount(recs[:, k], minlength=counts.shape[0])
    assert np.array_equal(got.astype(np.uint64), counts)


def test_motif_listing_hub_graph_and_query():
    """A graph with a hub (larger neighbourhoods than a warp, hand-offs
    between warps) and the query form: one pattern's subgraphs only."""
    g = G.disjoint_union(G.star(150), G.gnp(120, 0.06, 41), G.cycle(9))
    g = G.from_edges(g.n, np.concatenate([g.edges()[:, 0], np.arange(151, 171)]),
                     np.concatenate([g.edges()[:, 1], np.zeros(20, dtype=np.int64)]))
    k = 4
    dg = gpm.graph_from_csr(g)
    want = O.motif_count(g, k)
    A = _adj_matrix(g)
    col = Collect()
    n = gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, k, col, ring_records=512)
    recs = col.records(k)
    assert n == sum(want.values())
    assert _check_motifs(g, k, recs, A) == want
    counts = gpm.gpm_motif_count(dg, k)
    for p in range(gpm.gpm_motif_num_patterns(k)):
        col = Collect()
        n = gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, k, col, pattern=p, ring_records=128)
        recs = col.records(k)
        assert n == recs.shape[0] == int(counts[p])
        assert (recs[:, k] == p).all()
        if n:
            _check_motifs(g, k, recs, A)


def test_consumer_stop_and_exceptions():
    g = G.sbm(600, 60, 0.55, 0.01, 5)
    dg = gpm.graph_from_csr(g)
    total = gpm.gpm_clique_count(dg, 4)
    col = Collect(stop_after=2)
    n = gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, 4, col, ring_records=1024)
    assert 0 < n < total and n == col.records(4).shape[0]
    col = Collect(stop_after=1)
    n = gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, 4, col, ring_records=1024)
    assert n == col.records(4).shape[0] > 0

    def boom(recs):
        raise KeyError("consumer failed")

    with pytest.raises(KeyError):
        gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, 4, boom)
    # the graph is still usable, and a full listing afterwards is complete
    col = Collect()
    assert gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, 4, col) == total
    assert gpm.gpm_clique_count(dg, 4) == total


def test_slow_consumer_times_out_and_recovers():
    """The device waits for ring space at most max_idle_ms without host
    progress; a consumer that sleeps longer makes the wait run out."""
    g = G.sbm(600, 60, 0.55, 0.01, 5)
    dg = gpm.graph_from_csr(g)
    total = gpm.gpm_clique_count(dg, 4)
    gpm.gpm_set_config(dg, max_idle_ms=200)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, 4, Collect(sleep_first=1.0), ring_records=64)
    assert e.value.status == gpm.GPM_ETIMEOUT
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, 5, Collect(sleep_first=1.0), ring_records=64)
    assert e.value.status == gpm.GPM_ETIMEOUT
    gpm.gpm_set_config(dg, max_idle_ms=120000)
    col = Collect()
    assert gpm.gpm_list(gpm.graph_from_csr(g), gpm.GPM_APP_CLIQUE, 4, col, ring_records=64) == total
    col = Collect()
    assert gpm.gpm_list(dg, gpm.GPM_APP_CLIQUE, 4, col, ring_records=64) == total
    assert gpm.gpm_clique_count(dg, 4) == total
    m = gpm.gpm_motif_count(dg, 4)
    col = Collect()
    assert gpm.gpm_list(dg, gpm.GPM_APP_MOTIF, 4, col) == int(m.sum())


def test_listing_rejects_bad_arguments():
    dg = gpm.graph_from_csr(G.gnp(30, 0.2, 1))
    ok = Collect()
    bad = [(gpm.GPM_APP_CLIQUE, 2, -1, 0), (gpm.GPM_APP_CLIQUE, 17, -1, 0), (gpm.GPM_APP_CLIQUE, 4, 0, 0),
           (gpm.GPM_APP_MOTIF, 9, -1, 0), (gpm.GPM_APP_MOTIF, 4, 6, 0), (gpm.GPM_APP_MOTIF, 4, -2, 0),
           (gpm.GPM_APP_MOTIF, 4, -1, 63), (7, 4, -1, 0)]
    for app, k, pat, ring in bad:
        with pytest.raises(gpm.GpmError) as e:
            gpm.gpm_list(dg, app, k, ok, pattern=pat, ring_records=ring)
        assert e.value.status == gpm.GPM_EINVAL, (app, k, pat, ring)
    assert ok.calls == 0
