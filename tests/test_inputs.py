"""The synthetic workloads against their recipes (CPU).

Every stored oracle value under tests/golden/ names the sha256 of the graph
it was computed on; the generators must reproduce those bytes on any host
(the GPU tests and the benchmark regenerate the graphs there), and each
graph must have the shape its recipe states: size, degree structure, the
CSR conventions the library requires (sorted, symmetric, no self-loops or
repeated edges).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

from paper_2212_04551_gb300 import graphs as G

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _stored_sha(name):
    with open(os.path.join(GOLDEN, f"{name}.json")) as f:
        return json.load(f)["sha256"]


def _check_csr(g):
    ip, ix = g.indptr, g.indices
    assert ip.dtype == np.int32 and ix.dtype == np.int32
    assert ip[0] == 0 and ip[-1] == ix.shape[0] and (np.diff(ip) >= 0).all()
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(ip))
    assert (ix >= 0).all() and (ix < g.n).all()
    assert (src != ix).all(), "self-loop"
    # sorted and without repeats inside every list
    same_row = src[1:] == src[:-1]
    assert (ix[1:][same_row] > ix[:-1][same_row]).all()
    # symmetric: the reversed arcs are the same set
    fwd = src * g.n + ix
    rev = ix.astype(np.int64) * g.n + src
    assert np.array_equal(np.sort(fwd), np.sort(rev))


@pytest.mark.parametrize("name", ["er516", "rmat16", "sbm2000"])
def test_small_workloads_reproduce_stored_bytes(name):
    g = G.workload(name)
    assert g.sha256() == _stored_sha(name)
    _check_csr(g)


def test_er516_recipe():
    g = G.workload("er516")
    assert g.n == 516 and g.edges().shape[0] == 1200


def test_rmat16_recipe():
    g = G.workload("rmat16")
    d = g.degrees()
    assert g.n == 1 << 16
    assert g.edges().shape[0] == 477_873
    assert int(d.argmax()) == 0 and int(d.max()) == 6_444   # MSB-first quadrants: the hub is vertex 0


def test_sbm2000_recipe():
    g = G.workload("sbm2000")
    e = g.edges()
    assert g.n == 2000
    inside = (e[:, 0] // 100) == (e[:, 1] // 100)
    # 20 blocks of 100: p_in 0.5 on 20 * 4,950 pairs, p_out 0.01 on the rest
    n_in, n_out = 20 * 4950, 2000 * 1999 // 2 - 20 * 4950
    assert abs(inside.sum() / n_in - 0.5) < 0.01
    assert abs((~inside).sum() / n_out - 0.01) < 0.001


def test_chunglu1m_recipe_and_bytes():
    g = G.workload("chunglu1m")
    assert g.sha256() == _stored_sha("chunglu1m")
    d = g.degrees()
    assert g.n == 1_000_000 and g.edges().shape[0] == 7_544_878
    assert 14.0 < d.mean() < 16.5            # mean expected degree 16, less the merged repeats
    assert int(d.max()) <= 20_000            # expected degrees capped at 20,000
    # heavy tail: degrees above 100 exist, and the top 1 % of vertices hold
    # far more than 1 % of the edge ends
    top = np.sort(d)[-10_000:]
    assert int(d.max()) > 1000 and top.sum() > 0.15 * d.sum()


def test_ba4096_recipe_and_bytes():
    gs = G.workload("ba4096")
    assert len(gs) == 4096
    h = hashlib.sha256()
    for g in gs:
        h.update(g.sha256().encode())
    assert h.hexdigest() == _stored_sha("ba4096")
    ns = np.array([g.n for g in gs])
    assert ns.min() >= 20 and ns.max() <= 400
    for g in gs[:64]:
        _check_csr(g)
        d = g.degrees()
        # attachment m in [2, 6]: every vertex after the seed has >= 2 edges
        assert d.min() >= 1 and np.median(d) >= 2
