"""gpm_motif_count_noalloc: the allocation-free entry point.

It serves callers that cannot let a library allocate device memory (hosts
that own every device byte through their own pool, or a fixed device-memory
budget).  Checked here through the C ABI, on two calls in a row (the second
call finds the scratch array holding the first call's contents):

* against the CPU oracle (per pattern, by canonical code) and against the
  allocating entry point gpm_motif_count on the same graph -- the counts are
  integers, so they must be equal;
* that a call after the first one takes no device memory: the device's free
  memory is the same before and after it.

This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu


def _device_csr(g):
    import torch
    return torch.from_numpy(g.indptr).cuda(), torch.from_numpy(g.indices).cuda()


def _graph(name):
    if name == "er516":
        return G.erdos_renyi_m(516, 1200, 0)
    if name == "gnp120":
        return G.gnp(120, 0.08, 31)
    if name == "gnp60":
        return G.gnp(60, 0.1, 32)
    return G.barabasi_albert_batch(1, 300, 300, 4, 4, seed=9)[0]


@pytest.mark.parametrize("name,k", [("er516", 4), ("er516", 5), ("gnp120", 3), ("gnp120", 6), ("ba", 5),
                                    ("gnp60", 7)])
def test_noalloc_matches_oracle_twice(name, k):
    import torch
    g = _graph(name)
    want = O.motif_count(g, k)
    ref = gpm.gpm_motif_count(gpm.graph_from_csr(g), k)
    ip, ix = _device_csr(g)
    stream = torch.cuda.current_stream()
    first = gpm.gpm_motif_count_noalloc(ip, ix, g.n, k, stream=stream)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    second = gpm.gpm_motif_count_noalloc(ip, ix, g.n, k, stream=stream)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, "the second call took device memory"
    for got in (first, second):
        assert {gpm.gpm_motif_pattern(k, p): int(c) for p, c in enumerate(got) if c} == want
        assert np.array_equal(got, ref)
    assert int(ref.sum()) > 0


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    g = G.path(9000)
    ip, ix = _device_csr(g)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_motif_count_noalloc(ip, ix, g.n, 4)
    assert e.value.status == gpm.GPM_EINVAL and "8192" in str(e.value)
    with pytest.raises(gpm.GpmError) as e:
        gpm.gpm_motif_count_noalloc(ip, ix, 100, 8)
    assert e.value.status == gpm.GPM_EINVAL
    assert torch.cuda.is_available()
