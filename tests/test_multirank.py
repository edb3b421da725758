"""Root sharding over ranks (world size 2, gloo, CPU): disjoint shards cover
every root once, and the summed per-rank counts equal the single-rank
counts.  The per-rank counting here is the oracle (no GPU needed); the GPU
path uses the same shards through gpm_count_roots."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2212_04551_gb300 import graphs as G
from paper_2212_04551_gb300 import shard


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = G.sbm(300, 30, 0.4, 0.03, 8)
    order = shard.heaviest_first(g.degrees())
    mine = shard.shard_roots(order, rank, world)
    cl = [O.clique_count(g, k, order=O.ORDER_DEGREE, roots=mine) for k in (3, 4, 5)]
    mo = O.motif_count(g, 4, roots=mine)
    codes = sorted(O.motif_count(g, 4))
    vec = cl + [mo.get(c, 0) for c in codes]
    total = shard.reduce_counts(vec)
    out[rank] = (mine.tolist(), total)
    dist.destroy_process_group()


def test_two_rank_root_sharding():
    from oracle import oracle as O
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    g = G.sbm(300, 30, 0.4, 0.03, 8)
    roots0, tot0 = out[0]
    roots1, tot1 = out[1]
    assert sorted(roots0 + roots1) == list(range(g.n))      # a partition of the roots
    assert tot0 == tot1
    full = [O.clique_count(g, k) for k in (3, 4, 5)]
    mo = O.motif_count(g, 4)
    assert tot0 == full + [mo[c] for c in sorted(mo)]


def test_shard_helpers():
    order = shard.heaviest_first(np.array([3, 9, 9, 1]))
    assert order.tolist() == [1, 2, 0, 3]
    assert shard.shard_roots(order, 1, 2).tolist() == [2, 3]
    with pytest.raises(ValueError):
        shard.shard_roots(order, 2, 2)
    assert shard.reduce_counts([1, 2]) == [1, 2]
