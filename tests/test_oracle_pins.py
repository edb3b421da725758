"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check is chosen so that a plausible slip in the oracle (a dropped filter,
a wrong comparison in "lower" or in the canonical test, a transposed bit in
the code, a missing relabeling) fails at least one of them:

* closed forms: C(n,k) cliques in K_n, e_k(part sizes) in Turan graphs,
  trace(A^3)/6 triangles, sum C(d,2) - 3T wedges, path/cycle/star/Petersen
  motif counts, the star identity;
* independent library routines: networkx clique enumeration, networkx
  isomorphism classes over brute-forced k-subsets, the networkx graph atlas;
* invariants: per-root sums, order independence, relabelling invariance,
  all induced k-subsets summing to C(n,k);
* the paper's k = 4 dictionary facts (Section 4.3.4) and the OEIS class
  counts stored under tests/golden/.
"""
from __future__ import annotations

import itertools
import os
from math import comb

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import graphs as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_classes():
    rows = {}
    with open(os.path.join(GOLDEN, "graph_classes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, c, a = (int(x) for x in line.split())
            rows[k] = (c, a)
    return rows


def _adj_matrix(g) -> np.ndarray:
    a = np.zeros((g.n, g.n), dtype=np.int64)
    e = g.edges()
    a[e[:, 0], e[:, 1]] = 1
    a[e[:, 1], e[:, 0]] = 1
    return a


def _elem_sym(vals, k):
    e = [1] + [0] * k
    for x in vals:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * x
    return e[k]


def _random_small(seed, n=None, p=None):
    rng = np.random.default_rng(1000 + seed)
    n = n or int(rng.integers(5, 14))
    p = p if p is not None else float(rng.uniform(0.15, 0.7))
    return G.gnp(n, p, seed)


# ------------------------------------------------------------------ cliques

@pytest.mark.parametrize("n", [1, 2, 5, 9, 13])
def test_clique_complete_graph(n):
    g = G.complete(n)
    for k in range(1, min(n + 2, 14)):
        assert O.clique_count(g, k) == comb(n, k)
        assert O.clique_count(g, k, order=O.ORDER_DEGREE) == comb(n, k)


def test_clique_empty_and_union():
    assert O.clique_count(G.empty(7), 1) == 7
    for k in range(2, 5):
        assert O.clique_count(G.empty(7), k) == 0
    g = G.disjoint_union(G.complete(6), G.complete(9), G.path(4))
    for k in range(3, 10):
        assert O.clique_count(g, k) == comb(6, k) + comb(9, k)
    assert O.clique_count(g, 2) == 15 + 36 + 3


@pytest.mark.parametrize("n,r", [(10, 3), (17, 4), (12, 12), (9, 2)])
def test_clique_turan(n, r):
    g = G.turan(n, r)
    parts = [len(range(i, n, r)) for i in range(r)]
    for k in range(1, r + 2):
        assert O.clique_count(g, k) == _elem_sym(parts, k)


@pytest.mark.parametrize("seed", range(6))
def test_triangles_trace(seed):
    g = _random_small(seed, n=40, p=0.3)
    a = _adj_matrix(g)
    t = int(np.trace(a @ a @ a)) // 6
    assert O.clique_count(g, 3) == t
    assert O.clique_count(g, 3, order=O.ORDER_DEGREE) == t


@pytest.mark.parametrize("seed", range(8))
def test_cliques_vs_networkx(seed):
    nx = pytest.importorskip("networkx")
    g = _random_small(seed, n=30, p=0.45)
    h = nx.Graph()
    h.add_nodes_from(range(g.n))
    h.add_edges_from(map(tuple, g.edges()))
    by_k: dict[int, int] = {}
    first: dict[tuple[int, int], int] = {}
    for c in nx.enumerate_all_cliques(h):
        by_k[len(c)] = by_k.get(len(c), 0) + 1
        key = (len(c), min(c))
        first[key] = first.get(key, 0) + 1
    for k in range(1, 9):
        assert O.clique_count(g, k) == by_k.get(k, 0)
        # per-root decomposition under the id order: root = smallest id
        tot, pr = O.clique_count(g, k, per_root=True)
        assert tot == by_k.get(k, 0)
        assert [int(x) for x in pr] == [first.get((k, v), 0) for v in range(g.n)]


@pytest.mark.parametrize("seed", range(4))
def test_clique_degree_order_per_root(seed):
    nx = pytest.importorskip("networkx")
    g = _random_small(seed, n=28, p=0.5)
    d = g.degrees()
    h = nx.Graph()
    h.add_nodes_from(range(g.n))
    h.add_edges_from(map(tuple, g.edges()))
    for k in (3, 4, 5):
        want = np.zeros(g.n, dtype=np.int64)
        for c in nx.enumerate_all_cliques(h):
            if len(c) == k:
                want[min(c, key=lambda v: (d[v], v))] += 1
        tot, pr = O.clique_count(g, k, order=O.ORDER_DEGREE, per_root=True)
        assert tot == int(want.sum())
        assert np.array_equal(pr.astype(np.int64), want)
        # a root subset returns exactly those roots' counts
        roots = np.arange(0, g.n, 3)
        tot_s, pr_s = O.clique_count(g, k, order=O.ORDER_DEGREE, roots=roots, per_root=True)
        assert tot_s == int(want[roots].sum())
        assert np.array_equal(pr_s.astype(np.int64), want[roots])


# -------------------------------------------------------- canonical codes

def _atlas_by_k():
    nx = pytest.importorskip("networkx")
    out: dict[int, list] = {}
    for h in nx.graph_atlas_g():
        out.setdefault(h.number_of_nodes(), []).append(h)
    return out


def test_canon_is_complete_invariant_atlas():
    """Distinct on non-isomorphic graphs, equal on relabelled copies, for every
    graph on up to 7 vertices (networkx atlas), and the class counts match
    OEIS A001349 / A000088."""
    nx = pytest.importorskip("networkx")
    golden = _golden_classes()
    rng = np.random.default_rng(7)
    atlas = _atlas_by_k()
    for k in range(1, 8):
        graphs = atlas[k]
        codes = [O.full_code(h.edges(), k) for h in graphs]
        canon = O.canon_many(k, codes)
        assert len(set(canon.tolist())) == len(graphs) == golden[k][1]
        n_conn = sum(1 for h in graphs if nx.is_connected(h))
        assert n_conn == golden[k][0]
        for h, c in zip(graphs, canon):
            assert O.code_connected(k, int(c)) == nx.is_connected(h)
        # relabelled copies
        sample = range(0, len(graphs), max(1, len(graphs) // 60))
        for i in sample:
            h = graphs[i]
            perm = rng.permutation(k)
            e = [(int(perm[a]), int(perm[b])) for a, b in h.edges()]
            assert O.canon(k, O.full_code(e, k)) == int(canon[i])


def test_oracle_class_enumeration_matches_oeis():
    golden = _golden_classes()
    for k in range(1, 7):
        assert len(O.classes(k, True)) == golden[k][0]
        assert len(O.classes(k, False)) == golden[k][1]


def test_paper_k4_dictionary():
    """Section 4.3.4: k = 4 traversal bitmaps have 5 bits (v0-v1 implicit),
    low two bits = v2's edges to (v0, v1), next three = v3's edges to
    (v0, v1, v2).  Of the 32 codes, those where v2 and v3 each have an
    earlier neighbour are connected traversals, and they reach exactly the
    connected 4-vertex classes."""
    meta = {}
    with open(os.path.join(GOLDEN, "paper_k4_dictionary.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            meta[key] = [int(v) for v in vals]
    assert meta["bits"] == [5] and meta["codes"] == [32]
    golden = _golden_classes()
    reps = set()
    valid = 0
    for t in range(meta["codes"][0]):
        v2 = [(0, 2), (1, 2)]
        v3 = [(0, 3), (1, 3), (2, 3)]
        e = [(0, 1)]
        e += [v2[b] for b in range(2) if (t >> b) & 1]
        e += [v3[b] for b in range(3) if (t >> (2 + b)) & 1]
        if (t & 0b11) == 0 or (t >> 2) == 0:
            continue
        valid += 1
        c = O.canon(4, O.full_code(e, 4))
        assert O.code_connected(4, c)
        reps.add(c)
    assert valid == 21
    assert len(reps) == golden[4][0] == 6


# ---------------------------------------------------------------- motifs

def _nx_motifs(g, k):
    """Brute force over k-subsets with networkx: {canonical code: count}."""
    nx = pytest.importorskip("networkx")
    h = nx.Graph()
    h.add_nodes_from(range(g.n))
    h.add_edges_from(map(tuple, g.edges()))
    reps: list = []
    counts: list[int] = []
    for s in itertools.combinations(range(g.n), k):
        sub = h.subgraph(s)
        if not nx.is_connected(sub):
            continue
        for i, r in enumerate(reps):
            if nx.is_isomorphic(sub, r):
                counts[i] += 1
                break
        else:
            reps.append(nx.convert_node_labels_to_integers(sub))
            counts.append(1)
    out = {}
    for r, c in zip(reps, counts):
        out[O.canon(k, O.full_code(r.edges(), k))] = c
    return out


@pytest.mark.parametrize("seed", range(10))
def test_motifs_vs_networkx_bruteforce(seed):
    g = _random_small(seed, n=11)
    for k in (2, 3, 4, 5):
        assert O.motif_count(g, k) == _nx_motifs(g, k)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_sums_to_binomial(seed):
    g = _random_small(seed, n=14)
    for k in (3, 4, 5, 6):
        bf = O.brute_force(g, k)
        assert sum(c for c, _ in bf.values()) == comb(g.n, k)
        conn = {code: c for code, (c, is_conn) in bf.items() if is_conn}
        assert conn == O.motif_count(g, k)
        full = (1 << (k * (k - 1) // 2)) - 1
        assert bf.get(full, (0, True))[0] == O.clique_count(g, k)


@pytest.mark.parametrize("seed", range(6))
def test_k3_wedges_and_triangles(seed):
    g = _random_small(seed, n=60, p=0.12)
    a = _adj_matrix(g)
    tri = int(np.trace(a @ a @ a)) // 6
    d = g.degrees()
    wedges = int(sum(comb(int(x), 2) for x in d)) - 3 * tri
    got = O.motif_count(g, 3)
    path3 = O.canon(3, O.full_code([(0, 1), (1, 2)], 3))
    tri3 = O.canon(3, O.full_code([(0, 1), (1, 2), (0, 2)], 3))
    assert got.get(path3, 0) == wedges
    assert got.get(tri3, 0) == tri


def _dominating(k, code):
    """vertices adjacent to all others in the k-graph with this full code"""
    adj = [[False] * k for _ in range(k)]
    for i in range(1, k):
        for j in range(i):
            if (code >> (i * (i - 1) // 2 + j)) & 1:
                adj[i][j] = adj[j][i] = True
    return sum(1 for v in range(k) if all(adj[v][u] for u in range(k) if u != v))


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_star_identity(k):
    """Every k-set containing a vertex and k-1 of its neighbours is connected,
    so sum_p dom(p) * count_p = sum_v C(d(v), k-1)."""
    g = G.sbm(120, 20, 0.35, 0.03, 11)
    got = O.motif_count(g, k)
    lhs = sum(_dominating(k, code) * c for code, c in got.items())
    rhs = sum(comb(int(x), k - 1) for x in g.degrees())
    assert lhs == rhs


def test_structured_motifs():
    star_k = lambda k: O.canon(k, O.full_code([(0, i) for i in range(1, k)], k))
    path_k = lambda k: O.canon(k, O.full_code([(i, i + 1) for i in range(k - 1)], k))
    cyc_k = lambda k: O.canon(k, O.full_code([(i, (i + 1) % k) for i in range(k)], k))
    for n in (5, 9, 15):
        for k in range(2, 7):
            if k <= n:
                assert O.motif_count(G.path(n), k) == {path_k(k): n - k + 1}
            if k < n:
                assert O.motif_count(G.cycle(n), k) == {path_k(k): n}
        assert O.motif_count(G.cycle(n), n if n <= 8 else 8) == (
            {cyc_k(n): 1} if n <= 8 else {path_k(8): n})
    for s in (3, 7, 12):
        for k in range(2, 7):
            want = comb(s, k - 1)
            assert O.motif_count(G.star(s), k) == ({star_k(k): want} if want else {})
    pet = O.motif_count(G.petersen(), 4)
    assert pet == {star_k(4): 10, path_k(4): 60}
    assert O.motif_count(G.petersen(), 3) == {path_k(3): 30}


@pytest.mark.parametrize("seed", range(4))
def test_relabel_invariance(seed):
    g = _random_small(seed, n=40, p=0.15)
    perm = np.random.default_rng(seed).permutation(g.n)
    h = G.relabel(g, perm)
    for k in (3, 4, 5):
        assert O.motif_count(g, k) == O.motif_count(h, k)
        assert O.clique_count(g, k) == O.clique_count(h, k)


def test_motif_per_root_sums():
    g = _random_small(3, n=50, p=0.12)
    for k in (3, 4, 5):
        full, pr = O.motif_count(g, k, per_root=True)
        assert int(pr.sum()) == sum(full.values())
        a = O.motif_count(g, k, roots=np.arange(0, 25))
        b = O.motif_count(g, k, roots=np.arange(25, 50))
        merged = dict(a)
        for c, v in b.items():
            merged[c] = merged.get(c, 0) + v
        assert merged == full


# ----------------------------------------- clique search-tree instrumentation

def _rank_key(g):
    d = g.degrees()
    return lambda v: (int(d[v]), int(v))


def _balg_bruteforce(g, k):
    """B_alg from its definition, with sets: for every clique S of size
    1..k-2, C(S) = vertices after all of S in the (degree, id) order and
    adjacent to all of S; each v in C(S) adds 4 (|C(S)| + d+(v))."""
    import networkx as nx
    key = _rank_key(g)
    adj = [set(g.indices[g.indptr[v]:g.indptr[v + 1]].tolist()) for v in range(g.n)]
    dplus = [sum(1 for x in adj[v] if key(x) > key(v)) for v in range(g.n)]
    nxg = nx.Graph()
    nxg.add_nodes_from(range(g.n))
    nxg.add_edges_from(g.edges().tolist())
    total = 0
    for S in nx.enumerate_all_cliques(nxg):
        if len(S) > k - 2:
            break
        top = max(key(v) for v in S)
        C = [v for v in range(g.n) if key(v) > top and all(v in adj[u] for u in S)]
        total += sum(4 * (len(C) + dplus[v]) for v in C)
    return total


@pytest.mark.parametrize("seed", range(6))
def test_clique_instrument_nodes_and_bytes(seed):
    """Nodes per size equal networkx's clique counts, and B_alg equals its
    set-based definition (a dropped level, a wrong candidate set or a wrong
    out-degree changes one of them)."""
    import networkx as nx
    rng = np.random.default_rng(70 + seed)
    g = G.gnp(int(rng.integers(8, 36)), float(rng.uniform(0.15, 0.6)), 300 + seed)
    k = 5
    r = O.clique_instrument(g, k)
    nxg = nx.Graph()
    nxg.add_nodes_from(range(g.n))
    nxg.add_edges_from(g.edges().tolist())
    by_size = [0] * (k + 1)
    for S in nx.enumerate_all_cliques(nxg):
        if len(S) > k:
            break
        by_size[len(S)] += 1
    assert r["nodes"][1:] == by_size[1:]
    assert r["b_alg"] == _balg_bruteforce(g, k)


def test_clique_instrument_complete_graph_closed_form():
    """K_n: nodes[s] = C(n, s); a node of size s whose last vertex has rank m
    (C(m, s-1) of them) has n-1-m candidates, and child v (rank > m) has
    d+(v) = n-1-v, so B_alg = sum_s sum_m C(m, s-1) sum_{v>m} 4 (2n-2-m-v)."""
    n, k = 14, 6
    r = O.clique_instrument(G.complete(n), k)
    assert r["nodes"][1:] == [comb(n, s) for s in range(1, k + 1)]
    want = sum(comb(m, s - 1) * sum(4 * ((n - 1 - m) + (n - 1 - v)) for v in range(m + 1, n))
               for s in range(1, k - 1) for m in range(n))
    assert r["b_alg"] == want


def test_clique_instrument_root_partition():
    """Per-root restriction: the roots split the tree (every clique has one
    first vertex), so node counts and bytes add up over a root partition."""
    g = G.gnp(40, 0.35, 9)
    whole = O.clique_instrument(g, 5)
    roots = np.arange(g.n, dtype=np.int32)
    a = O.clique_instrument(g, 5, roots=roots[::2])
    b = O.clique_instrument(g, 5, roots=roots[1::2])
    assert [x + y for x, y in zip(a["nodes"], b["nodes"])] == whole["nodes"]
    assert a["b_alg"] + b["b_alg"] == whole["b_alg"]


# ------------------------------------------------ the ESU route of the oracle

@pytest.mark.parametrize("seed", range(8))
def test_esu_route_matches_bruteforce_and_arabesque(seed):
    """The oracle's ESU route (used for full-size stored values) against
    brute force over every k-subset (its connected classes) and against the
    Arabesque-filtered route, per pattern and per root."""
    g = _random_small(seed, n=14)
    for k in (1, 2, 3, 4, 5, 6):
        esu = O.motif_count(g, k, method="esu")
        bf = {code: c for code, (c, conn) in O.brute_force(g, k).items() if conn}
        assert esu == bf, k
    rng = np.random.default_rng(90 + seed)
    h = G.gnp(int(rng.integers(20, 60)), float(rng.uniform(0.05, 0.3)), 400 + seed)
    roots = np.arange(h.n, dtype=np.int32)[::3]
    for k in (3, 4, 5):
        a, pa = O.motif_count(h, k, roots=roots, per_root=True)
        b, pb = O.motif_count(h, k, roots=roots, per_root=True, method="esu")
        assert a == b and np.array_equal(pa, pb), k


def test_esu_route_structured_graphs():
    """Closed forms: K_n has C(n,k) sets, all cliques; the star K_{1,s} has
    C(s, k-1) induced stars; the path P_n has n-k+1 induced paths."""
    for k in (3, 4, 5):
        assert O.motif_count(G.complete(9), k, method="esu") == {(1 << (k * (k - 1) // 2)) - 1: comb(9, k)}
        star = O.motif_count(G.star(12), k, method="esu")
        assert sum(star.values()) == comb(12, k - 1) and len(star) == 1
        path = O.motif_count(G.path(15), k, method="esu")
        assert sum(path.values()) == 15 - k + 1 and len(path) == 1


# ------------------------------------------------ the bitset route of the oracle

def test_bits_route_complete_graph_closed_form():
    """K_n with out-neighbourhoods wider than one 64-bit word: C(n, s)."""
    for n in (1, 2, 9, 70, 131):
        c = O.clique_count_bits(G.complete(n), 5)
        assert c[1:] == [comb(n, s) for s in range(1, 6)]


@pytest.mark.parametrize("n,r", [(17, 4), (150, 10), (12, 12), (9, 2)])
def test_bits_route_turan(n, r):
    g = G.turan(n, r)
    parts = [len(range(i, n, r)) for i in range(r)]
    k = min(r + 1, 7)
    c = O.clique_count_bits(g, k)
    assert c[1:] == [_elem_sym(parts, s) for s in range(1, k + 1)]


def test_bits_route_empty_and_union():
    g = G.disjoint_union(G.complete(6), G.complete(70), G.path(4), G.empty(3))
    c = O.clique_count_bits(g, 6)
    assert c[1] == g.n and c[2] == g.m
    for s in range(3, 7):
        assert c[s] == comb(6, s) + comb(70, s)


@pytest.mark.parametrize("seed", range(4))
def test_bits_route_vs_networkx_per_root(seed):
    """Per size and per root (root = first vertex in the (degree, id)
    order): networkx's cliques, counted by their lowest-ranked vertex."""
    nx = pytest.importorskip("networkx")
    g = _random_small(seed, n=34, p=0.5)
    d = g.degrees()
    h = nx.Graph()
    h.add_nodes_from(range(g.n))
    h.add_edges_from(map(tuple, g.edges()))
    k = 7
    want = np.zeros((g.n, k + 1), dtype=np.int64)
    for c in nx.enumerate_all_cliques(h):
        if len(c) <= k:
            want[min(c, key=lambda v: (d[v], v)), len(c)] += 1
    counts, pr = O.clique_count_bits(g, k, per_root=True)
    assert counts[1:] == [int(x) for x in want.sum(axis=0)[1:]]
    assert np.array_equal(pr[:, 1:].astype(np.int64), want[:, 1:])
    roots = np.arange(1, g.n, 3, dtype=np.int32)
    counts_s, pr_s = O.clique_count_bits(g, k, roots=roots, per_root=True)
    assert counts_s[1:] == [int(x) for x in want[roots].sum(axis=0)[1:]]
    assert np.array_equal(pr_s[:, 1:].astype(np.int64), want[roots, 1:])


@pytest.mark.parametrize("seed", range(3))
def test_clique_routes_on_joins(seed):
    """The join a + b (all edges between a and b added): every clique of it
    is a clique of a beside a clique of b, so its k-cliques number
    sum_i c_i(a) c_{k-i}(b) with c_0 = 1.  The parts' counts come from
    networkx; both clique routes must give the join's."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(900 + seed)
    a = G.gnp(int(rng.integers(8, 30)), float(rng.uniform(0.1, 0.6)), 910 + seed)
    b = G.gnp(int(rng.integers(5, 25)), float(rng.uniform(0.1, 0.6)), 920 + seed)
    k_hi = 7

    def nx_counts(g):
        h = nx.Graph()
        h.add_nodes_from(range(g.n))
        h.add_edges_from(map(tuple, g.edges()))
        c = [1] + [0] * k_hi
        for q in nx.enumerate_all_cliques(h):
            if len(q) <= k_hi:
                c[len(q)] += 1
        return c

    ca, cb = nx_counts(a), nx_counts(b)
    want = [sum(ca[i] * cb[k - i] for i in range(k + 1)) for k in range(k_hi + 1)]
    j = G.join(a, b)
    assert O.clique_count_bits(j, k_hi)[1:] == want[1:]
    for k in (3, 5, 7):
        assert O.clique_count(j, k) == want[k]


@pytest.mark.parametrize("seed", range(3))
def test_bits_route_vs_list_route_wide_rows(seed):
    """Out-neighbourhoods of 60-200 vertices (rows of 1-4 words): the same
    per-root counts as the sorted-list route of Algorithm 4 in the (degree,
    id) order, which the closed forms and networkx pin above."""
    g = G.gnp(260, 0.42 + 0.05 * seed, 500 + seed)
    roots = np.arange(0, g.n, 7, dtype=np.int32)
    counts, pr = O.clique_count_bits(g, 5, roots=roots, per_root=True)
    for k in (3, 4, 5):
        tot, want = O.clique_count(g, k, order=O.ORDER_DEGREE, roots=roots, per_root=True)
        assert counts[k] == tot
        assert np.array_equal(pr[:, k], want)
