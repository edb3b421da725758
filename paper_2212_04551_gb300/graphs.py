"""Seeded synthetic input graphs, shared by the tests, the benchmark and the oracle.

This module holds no part of the enumeration method: it only draws random
graphs and packs them as undirected int32 CSR (``indptr[n+1]``, ``indices``),
every adjacency list sorted ascending, symmetric, with no self-loops and no
duplicate edges -- the input format the paper assumes (Section 2: undirected,
unlabelled graphs; Section 4.3.1: each adjacency list contiguous in memory).

The paper evaluates on five real graphs (Table 2: Citeseer, ca-AstroPh, Mico,
com-DBLP, com-LiveJournal), none of which is available here.  The generators
below are the synthetic stand-ins, every one driven by ``numpy.random.
default_rng(seed)`` (PCG64) so that any machine rebuilds identical bytes:

* ``erdos_renyi_m``  -- G(n, m) by rejection of self-loops and repeats
  (516 vertices / 1,200 edges mirrors bio-diseasome from Section 1);
* ``chung_lu``       -- power-law expected degrees (heavy-tailed like
  LiveJournal: average degree 16, exponent 2.1, cap 20,000);
* ``rmat``           -- recursive-matrix graph, hub kept at id 0 (root skew);
* ``barabasi_albert_batch`` -- thousands of small preferential-attachment graphs;
* ``sbm``            -- planted dense blocks (deep cliques);
* small structured graphs with closed-form counts (complete, path, cycle,
  star, Turan, Petersen, disjoint unions) used as pins.
"""
from __future__ import annotations

import functools
import hashlib
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CSR:
    """Undirected graph as int32 CSR; ``indices[indptr[v]:indptr[v+1]]`` = N(v)."""

    indptr: np.ndarray
    indices: np.ndarray

    @property
    def n(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return int(self.indices.shape[0] // 2)

    def degrees(self) -> np.ndarray:
        return np.diff(self.indptr).astype(np.int64)

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(self.indptr, dtype="<i4").tobytes())
        h.update(np.ascontiguousarray(self.indices, dtype="<i4").tobytes())
        return h.hexdigest()

    def edges(self) -> np.ndarray:
        """Each undirected edge once, as rows (u, v) with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.indptr))
        dst = self.indices.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)


def from_edges(n: int, u, v) -> CSR:
    """Symmetrise, drop self-loops and duplicates, sort: the canonical CSR."""
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    if u.size:
        if u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n:
            raise ValueError("edge endpoint out of range")
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = np.unique(a * n + b) if a.size else np.zeros(0, dtype=np.int64)
    src = key // n if n else key
    dst = key % n if n else key
    indptr = np.zeros(n + 1, dtype=np.int64)
    if n:
        np.cumsum(np.bincount(src, minlength=n), out=indptr[1:])
    if indptr[-1] >= 2**31:
        raise ValueError("more than 2^31-1 adjacency entries")
    return CSR(indptr.astype(np.int32), dst.astype(np.int32))


def relabel(g: CSR, perm: np.ndarray) -> CSR:
    """The same graph with vertex v renamed perm[v]."""
    e = g.edges()
    perm = np.asarray(perm, dtype=np.int64)
    return from_edges(g.n, perm[e[:, 0]], perm[e[:, 1]])


def disjoint_union(*gs: CSR) -> CSR:
    us, vs, off = [], [], 0
    for g in gs:
        e = g.edges()
        us.append(e[:, 0] + off)
        vs.append(e[:, 1] + off)
        off += g.n
    if not us:
        return from_edges(0, [], [])
    return from_edges(off, np.concatenate(us), np.concatenate(vs))


def join(a: CSR, b: CSR) -> CSR:
    """The join a + b: a and b side by side (b's vertices shifted by a.n),
    plus every edge between a vertex of a and a vertex of b."""
    ea, eb = a.edges(), b.edges()
    ia = np.repeat(np.arange(a.n, dtype=np.int64), b.n)
    ib = np.tile(np.arange(b.n, dtype=np.int64), a.n) + a.n
    return from_edges(a.n + b.n, np.concatenate([ea[:, 0], eb[:, 0] + a.n, ia]),
                      np.concatenate([ea[:, 1], eb[:, 1] + a.n, ib]))


# ---------------------------------------------------------------- structured

def empty(n: int) -> CSR:
    return from_edges(n, [], [])


def complete(n: int) -> CSR:
    iu = np.triu_indices(n, 1)
    return from_edges(n, iu[0], iu[1])


def path(n: int) -> CSR:
    a = np.arange(max(n - 1, 0))
    return from_edges(n, a, a + 1)


def cycle(n: int) -> CSR:
    a = np.arange(n)
    return from_edges(n, a, (a + 1) % n)


def star(s: int) -> CSR:
    """K_{1,s}: hub 0 joined to leaves 1..s."""
    return from_edges(s + 1, np.zeros(s, dtype=np.int64), np.arange(1, s + 1))


def turan(n: int, r: int) -> CSR:
    """Complete r-partite graph on n vertices with near-equal parts (v in part v % r)."""
    iu = np.triu_indices(n, 1)
    keep = (iu[0] % r) != (iu[1] % r)
    return from_edges(n, iu[0][keep], iu[1][keep])


def petersen() -> CSR:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(10, e[:, 0], e[:, 1])


def gnp(n: int, p: float, seed: int) -> CSR:
    """Each of the n(n-1)/2 pairs independently with probability p."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].shape[0]) < p
    return from_edges(n, iu[0][keep], iu[1][keep])


# ---------------------------------------------------------- paper stand-ins

def erdos_renyi_m(n: int = 516, m: int = 1200, seed: int = 0) -> CSR:
    """G(n, m): draw ``rng.integers(0, n, 2)`` pairs, skipping self-loops and
    pairs already present, until m distinct edges exist."""
    rng = np.random.default_rng(seed)
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds n(n-1)/2")
    seen: set[tuple[int, int]] = set()
    us, vs = [], []
    while len(seen) < m:
        a, b = (int(x) for x in rng.integers(0, n, 2))
        if a == b:
            continue
        key = (min(a, b), max(a, b))
        if key in seen:
            continue
        seen.add(key)
        us.append(key[0])
        vs.append(key[1])
    return from_edges(n, us, vs)


def chung_lu(n: int = 1_000_000, avg_deg: float = 16.0, gamma: float = 2.1,
             max_deg: float = 20_000.0, seed: int = 1, n_pairs: int | None = None) -> CSR:
    """Chung-Lu power law: weights w_i = (i+1)^(-1/(gamma-1)), rescaled to the
    target mean and capped (50 rounds of scale-then-cap), then ``n_pairs``
    endpoint pairs drawn i.i.d. proportional to w (u first, then v).  The
    default draws n*avg_deg/2 pairs (8,000,000 for the default n)."""
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (gamma - 1.0))
    for _ in range(50):
        w *= avg_deg / w.mean()
        np.minimum(w, max_deg, out=w)
    p = w / w.sum()
    if n_pairs is None:
        n_pairs = int(round(n * avg_deg / 2))
    u = rng.choice(n, size=n_pairs, p=p)
    v = rng.choice(n, size=n_pairs, p=p)
    return from_edges(n, u, v)


def rmat(scale: int = 16, edge_factor: int = 8, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 2) -> CSR:
    """R-MAT: 2^scale vertices, edge_factor*2^scale sampled edges; each edge
    descends ``scale`` levels most-significant bit first, picking quadrant
    (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, 1-a-b-c.  No noise
    and no vertex permutation, so the heaviest hub keeps id 0."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    ne = edge_factor * n
    u = np.zeros(ne, dtype=np.int64)
    v = np.zeros(ne, dtype=np.int64)
    for _ in range(scale):
        r = rng.random(ne)
        ubit = (r >= a + b).astype(np.int64)
        vbit = (((r >= a) & (r < a + b)) | (r >= a + b + c)).astype(np.int64)
        u = (u << 1) | ubit
        v = (v << 1) | vbit
    return from_edges(n, u, v)


def sbm(n: int = 2000, block: int = 100, p_in: float = 0.5, p_out: float = 0.01,
        seed: int = 4) -> CSR:
    """Stochastic block model, block(i) = i // block; one ``rng.random`` draw
    per pair i < j in row-major order of the upper triangle."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    r = rng.random(iu[0].shape[0])
    same = (iu[0] // block) == (iu[1] // block)
    keep = np.where(same, r < p_in, r < p_out)
    return from_edges(n, iu[0][keep], iu[1][keep])


def barabasi_albert(n: int, m_a: int, rng: np.random.Generator) -> CSR:
    """Preferential attachment: seed vertices 0..m_a-1 (no edges); vertex m_a
    joins all seeds; every later vertex picks m_a distinct targets with
    probability proportional to degree (uniform draws from the list of edge
    endpoints, redrawing duplicates)."""
    us: list[int] = []
    vs: list[int] = []
    ends: list[int] = []
    for t in range(m_a):
        us.append(m_a)
        vs.append(t)
        ends.extend((m_a, t))
    for new in range(m_a + 1, n):
        chosen: list[int] = []
        while len(chosen) < m_a:
            t = ends[int(rng.integers(0, len(ends)))]
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            us.append(new)
            vs.append(t)
            ends.extend((new, t))
    return from_edges(n, us, vs)


def barabasi_albert_batch(count: int = 4096, n_lo: int = 20, n_hi: int = 400,
                          m_lo: int = 2, m_hi: int = 6, seed: int = 3) -> list[CSR]:
    """``count`` BA graphs; per graph (in order) n ~ U[n_lo, n_hi] and
    m_a ~ U[m_lo, m_hi] (inclusive) drawn with ``rng.integers``, then the
    graph from the same generator."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        m_a = int(rng.integers(m_lo, m_hi + 1))
        out.append(barabasi_albert(n, m_a, rng))
    return out


def pack(graphs: list[CSR]) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Concatenate graphs: (graph_offsets[G+1] over vertices, indptr[N+1]
    global edge offsets, indices local to each graph)."""
    goff = np.zeros(len(graphs) + 1, dtype=np.int64)
    goff[1:] = np.cumsum([g.n for g in graphs])
    eoff = 0
    ip = [np.zeros(1, dtype=np.int64)]
    ind = []
    for g in graphs:
        ip.append(g.indptr[1:].astype(np.int64) + eoff)
        ind.append(g.indices)
        eoff += g.indices.shape[0]
    indptr = np.concatenate(ip)
    indices = np.concatenate(ind) if ind else np.zeros(0, dtype=np.int32)
    return goff.astype(np.int32), indptr.astype(np.int32), indices.astype(np.int32)


def sample_roots(n: int, count: int, seed: int, exclude=None) -> np.ndarray:
    """A seeded, sorted sample of ``count`` distinct root ids from [0, n)
    (all of them when count >= the eligible set); ``exclude`` is a boolean
    mask of ineligible vertices."""
    rng = np.random.default_rng(seed)
    pool = np.arange(n, dtype=np.int64)
    if exclude is not None:
        pool = pool[~np.asarray(exclude, dtype=bool)]
    if count >= pool.shape[0]:
        return pool.astype(np.int32)
    return np.sort(rng.choice(pool, size=count, replace=False)).astype(np.int32)


# Workloads used by the tests and the benchmark, named by what they are
# (cached in-process: the graphs are immutable once built).
@functools.lru_cache(maxsize=8)
def workload(name: str):
    if name == "er516":
        return erdos_renyi_m(516, 1200, 0)
    if name == "chunglu1m":
        return chung_lu(1_000_000, 16.0, 2.1, 20_000.0, 1)
    if name == "rmat16":
        return rmat(16, 8, 0.57, 0.19, 0.19, 2)
    if name == "ba4096":
        return tuple(barabasi_albert_batch(4096, 20, 400, 2, 6, 3))
    if name == "sbm2000":
        return sbm(2000, 100, 0.5, 0.01, 4)
    raise KeyError(name)
