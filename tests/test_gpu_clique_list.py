"""Clique counting on graphs with oriented out-degrees above the bitmap
limit of 1,024: the roots above it are counted by list intersection (the
extension step's array form), the others by the bitmap kernel, in one call.

Pins, none of them from the CUDA path:

* K_n: C(n, k); Turan graphs: e_k(part sizes);
* the join a + b of two sparse random graphs (every vertex of a adjacent to
  every vertex of b): a clique of the join is a clique of a beside a clique
  of b, so c_k(a + b) = sum_i c_i(a) c_{k-i}(b) (c_0 = 1), with the parts'
  counts from the CPU oracle (milliseconds: the parts are sparse);
* per root, on heavy and light roots of the join: the CPU oracle's bitset
  route.
"""
from __future__ import annotations

import functools
from math import comb

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu
LIMIT = 1024


@pytest.fixture(scope="module", autouse=True)
def _lib():
    gpm.load()
    O.build()


def _outdeg(g):
    """Out-degrees of the (degree, id) orientation."""
    d = g.degrees().astype(np.int64)
    e = g.edges()
    a, b = e[:, 0], e[:, 1]
    fwd = (d[a] < d[b]) | ((d[a] == d[b]) & (a < b))
    return np.bincount(np.where(fwd, a, b), minlength=g.n)


def _elem_sym(parts, s):
    e = [1] + [0] * s
    for x in parts:
        for j in range(s, 0, -1):
            e[j] += e[j - 1] * x
    return e[s]


@functools.lru_cache(maxsize=None)
def _join():
    a, b = G.gnp(1100, 0.05, 1), G.gnp(1100, 0.05, 2)
    return a, b, G.join(a, b)


def _join_counts(a, b, k_hi):
    ca = O.clique_count_bits(a, k_hi)
    cb = O.clique_count_bits(b, k_hi)
    c = lambda x, i: 1 if i == 0 else int(x[i])
    return [sum(c(ca, i) * c(cb, k - i) for i in range(k + 1)) for k in range(k_hi + 1)]


def test_complete_graph_above_the_limit():
    g = G.complete(1100)
    assert _outdeg(g).max() > LIMIT
    dg = gpm.graph_from_csr(g)
    for k in (3, 4):
        assert gpm.gpm_clique_count(dg, k) == comb(1100, k), k
    assert gpm.gpm_get_stats(dg)["kernel_launches"] >= 4   # bitmap launch + the list path's two
    assert gpm.gpm_clique_count_range(dg, 3, 4) == [comb(1100, 3), comb(1100, 4)]
    for k in (1, 2):
        assert gpm.gpm_clique_count(dg, k) == comb(1100, k)


def test_turan_graph_above_the_limit():
    n, r = 1300, 13
    g = G.turan(n, r)
    assert (_outdeg(g) > LIMIT).sum() > 100
    parts = [len(range(i, n, r)) for i in range(r)]
    dg = gpm.graph_from_csr(g)
    assert gpm.gpm_clique_count_range(dg, 3, 4) == [_elem_sym(parts, 3), _elem_sym(parts, 4)]


def test_join_matches_the_join_identity():
    a, b, j = _join()
    od = _outdeg(j)
    assert od.max() > LIMIT and (od > LIMIT).sum() > 100 and (od <= LIMIT).sum() > 100
    want = _join_counts(a, b, 8)
    dg = gpm.graph_from_csr(j)
    for k in range(3, 9):
        assert gpm.gpm_clique_count(dg, k) == want[k], k
    assert gpm.gpm_clique_count_range(dg, 3, 8) == want[3:9]
    assert gpm.gpm_clique_count_range(dg, 5, 6) == want[5:7]


def test_join_per_root_matches_oracle():
    """Per root, heavy and light roots mixed, against the oracle's bitset
    route; also the whole vertex set's per-root array sums to the total."""
    _, _, j = _join()
    od = _outdeg(j)
    rng = np.random.default_rng(7)
    heavy = rng.choice(np.flatnonzero(od > LIMIT), 10, replace=False)
    light = rng.choice(np.flatnonzero(od <= LIMIT), 10, replace=False)
    roots = np.concatenate([heavy, light]).astype(np.int32)
    rng.shuffle(roots)
    dg = gpm.graph_from_csr(j)
    for k in (4, 5):
        tot, want = O.clique_count_bits(j, k, roots=roots, per_root=True)
        c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, roots, per_root=True)
        assert int(c[0]) == tot[k], k
        assert np.array_equal(pr.astype(np.int64), want[:, k].astype(np.int64)), k
    c, pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, 5, None, per_root=True)
    assert int(pr.sum()) == int(c[0]) == gpm.gpm_clique_count(dg, 5)
    assert pr[od > LIMIT].sum() > 0 and pr[od <= LIMIT].sum() > 0


def test_join_schedules_and_monitored_balancing():
    """Pre-split schedules (heavy roots among the split ones) and the
    host-monitored form give the same counts, root by root."""
    torch = pytest.importorskip("torch")
    _, _, j = _join()
    od = _outdeg(j)
    dg = gpm.graph_from_csr(j)
    k = 5
    ref, ref_pr = gpm.gpm_count_roots(dg, gpm.GPM_APP_CLIQUE, k, None, per_root=True)
    scores = torch.from_numpy(od.astype(np.float32)).cuda()
    roots = np.arange(j.n, dtype=np.int32)
    for ns, ch in [(64, 8), (300, 2)]:
        gpm.gpm_sched_from_scores(dg, gpm.GPM_APP_CLIQUE, scores, roots, ns, ch)
        c, pr = gpm.gpm_count_scheduled(dg, gpm.GPM_APP_CLIQUE, k, n_roots=j.n, per_root=True)
        assert np.array_equal(c, ref) and np.array_equal(pr, ref_pr), (ns, ch)
    gpm.gpm_sched_balanced(dg, gpm.GPM_APP_CLIQUE, scores, roots, 8192, 64)
    c, pr = gpm.gpm_count_scheduled(dg, gpm.GPM_APP_CLIQUE, k, n_roots=j.n, per_root=True)
    assert np.array_equal(c, ref) and np.array_equal(pr, ref_pr)
    for threshold in (0.0, 0.4):
        cm, _ = gpm.gpm_count_monitored(dg, gpm.GPM_APP_CLIQUE, k, threshold)
        assert int(cm[0]) == int(ref[0]), threshold
    gpm.gpm_set_config(dg, donate=0)
    assert gpm.gpm_clique_count(dg, k) == int(ref[0])


def test_dm_dfs_above_the_limit():
    """The DM_DFS baseline (merged lists, no limit) agrees on the join."""
    a, b, j = _join()
    dg = gpm.graph_from_csr(j)
    assert gpm.gpm_clique_count_dfs(dg, 4) == _join_counts(a, b, 4)[4]
