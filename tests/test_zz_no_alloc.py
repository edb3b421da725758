"""gpm_motif_count_noalloc: the allocation-free entry point.

It serves callers that cannot let a library allocate device memory (hosts
that own every device byte through their own pool, or a fixed device-memory
budget).  Checked here through the C ABI against the allocating entry point
gpm_motif_count on the same graphs: the counts are integers, so they must be
equal, on two calls in a row (the second call finds the scratch array holding
the first call's contents).  This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2212_04551_gb300 import gpm
from paper_2212_04551_gb300 import graphs as G

pytestmark = pytest.mark.gpu


def _device_csr(g):
    import torch
    return torch.from_numpy(g.indptr).cuda(), torch.from_numpy(g.indices).cuda()


@pytest.mark.parametrize("name,k", [("er516", 4), ("er516", 5), ("gnp", 3), ("gnp", 6), ("ba", 5)])
def test_noalloc_matches_allocating_entry_twice(name, k):
    import torch
    if name == "er516":
        g = G.erdos_renyi_m(516, 1200, 0)
    elif name == "gnp":
        g = G.gnp(120, 0.08, 31)
    else:
        g = G.barabasi_albert_batch(1, 300, 300, 4, 4, seed=9)[0]
    ref = gpm.gpm_motif_count(gpm.graph_from_csr(g), k)
    ip, ix = _device_csr(g)
    stream = torch.cuda.current_stream()
    first = gpm.gpm_motif_count_noalloc(ip, ix, g.n, k, stream=stream)
    second = gpm.gpm_motif_count_noalloc(ip, ix, g.n, k, stream=stream)
    assert np.array_equal(first, ref)
    assert np.array_equal(second, ref)
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
