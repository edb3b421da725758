"""The identity behind the clique kernel's non-edge count (CPU check).

Below a child of a three-level tail node, the kernel counts the triangles
of G[X] (X = the child's candidates) as

    sum_t C(a_t, 2)  -  sum over non-adjacent u < v in X of |{t in X : t < u, t ~ u, t ~ v}|,

a_t = the neighbours of t above t inside X (vertices in the kernel's
orientation order).  The first sum counts each triangle once at its lowest
vertex plus each wedge u - t - v (t below u < v) whose ends are not
adjacent; the second counts those wedges from the non-edge side.  Checked
here against brute force on random graphs of every density, on complete
graphs (no non-edges) and on empty ones, with X a random subset, so that a
mistake in which side of t the wedge apex lies, or in which pairs are
non-edges, fails.
"""
from __future__ import annotations

from itertools import combinations
from math import comb

import numpy as np
import pytest


def _brute_triangles(A, X):
    return sum(1 for a, b, c in combinations(X, 3) if A[a, b] and A[a, c] and A[b, c])


def _identity(A, X):
    X = sorted(X)
    inX = set(X)
    P = Q = 0
    for t in X:
        a = sum(1 for u in X if u > t and A[t, u])
        P += comb(a, 2)
    for u, v in combinations(X, 2):          # u < v
        if A[u, v]:
            continue
        Q += sum(1 for t in X if t < u and A[t, u] and A[t, v])
    assert P >= Q
    return P - Q


def _random_graph(rng, n, p):
    A = np.zeros((n, n), dtype=bool)
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].shape[0]) < p
    A[iu[0][keep], iu[1][keep]] = True
    return A | A.T


@pytest.mark.parametrize("p", [0.0, 0.1, 0.5, 0.85, 0.97, 1.0])
def test_nonedge_triangle_identity(p):
    rng = np.random.default_rng(int(p * 1000) + 7)
    for _ in range(30):
        n = int(rng.integers(3, 40))
        A = _random_graph(rng, n, p)
        X = [v for v in range(n) if rng.random() < 0.8]
        assert _identity(A, X) == _brute_triangles(A, X)


def test_identity_on_complete_and_empty_sets():
    for n in (3, 10, 33):
        A = _random_graph(np.random.default_rng(n), n, 1.0)
        assert _identity(A, list(range(n))) == comb(n, 3)
        assert _identity(~A & ~np.eye(n, dtype=bool), list(range(n))) == 0


def test_identity_counts_each_open_wedge_once():
    # K_12 less one edge {9, 11}: the n - 2 triangles through it are gone,
    # 9 of them counted by the lower-apex wedges (t < 9) and removed by Q
    n = 12
    A = _random_graph(np.random.default_rng(1), n, 1.0)
    A[9, 11] = A[11, 9] = False
    X = list(range(n))
    assert _identity(A, X) == comb(n, 3) - (n - 2)
    assert _brute_triangles(A, X) == comb(n, 3) - (n - 2)


def _k4_from_nonedges(A, X):
    """#K4 of G[X] by inclusion-exclusion over the non-edges H of G[X]:
    every set F of non-edges spanning s <= 4 vertices enters with sign
    (-1)^|F| times the number of 4-sets containing them, C(c - s, 4 - s):
    no non-edge, one, two sharing a vertex (p3) or not, a triangle, a star
    or a path of three, and the sets of four or more on one 4-set."""
    X = sorted(X)
    c = len(X)
    H = {v: set() for v in X}
    for u, v in combinations(X, 2):
        if not A[u, v]:
            H[u].add(v)
            H[v].add(u)
    E = [(u, v) for u in X for v in H[u] if u < v]
    m = len(E)
    d = {v: len(H[v]) for v in X}
    p3 = sum(comb(d[v], 2) for v in X)                      # two non-edges sharing a vertex
    s3 = sum(comb(d[v], 3) for v in X)                      # three sharing one vertex
    tri = sum(1 for u, v in E for w in H[u] & H[v] if w > v)
    p4 = sum((d[u] - 1) * (d[v] - 1) for u, v in E) - 3 * tri
    # sets of 4, 5 or 6 non-edges (they span exactly 4 vertices): per 4-set
    # with e >= 4 non-edges among its vertices, its C(e, 4) - C(e, 5) + C(e, 6)
    # subsets -- a C4 or a paw counts once, a diamond (five non-edges)
    # 5 - 1 = 4 times (its C4, its four paws, less itself), a K4 15 - 6 + 1
    dense4 = 0
    for S in combinations(X, 4):
        e = sum(1 for a, b in combinations(S, 2) if b in H[a])
        if e >= 4:
            dense4 += comb(e, 4) - comb(e, 5) + comb(e, 6)
    return (comb(c, 4) - m * comb(c - 2, 2) + p3 * (c - 3) + (comb(m, 2) - p3)
            - tri * (c - 3) - s3 - p4 + dense4)


def _brute_k4(A, X):
    return sum(1 for S in combinations(sorted(X), 4) if all(A[a, b] for a, b in combinations(S, 2)))


@pytest.mark.parametrize("p", [0.0, 0.3, 0.5, 0.7, 0.9, 0.98, 1.0])
def test_k4_from_nonedges(p):
    """The next level's candidate: 4-cliques of a nearly complete candidate
    graph from its few non-edges (exact for every density)."""
    rng = np.random.default_rng(int(p * 100) + 11)
    for _ in range(12):
        n = int(rng.integers(4, 22))
        A = _random_graph(rng, n, p)
        X = [v for v in range(n) if rng.random() < 0.85]
        assert _k4_from_nonedges(A, X) == _brute_k4(A, X)
