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
