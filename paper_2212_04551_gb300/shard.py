"""Multi-GPU decomposition of the enumeration by roots (host logic only).

Every k-clique has exactly one root (its lowest-(degree, id) vertex) and every
connected induced k-subgraph has exactly one root (its smallest id), so the
roots partition the work: ranks count disjoint root sets with no exchange
during enumeration, and one sum of the per-rank count vectors (at most 853
uint64 for 7-vertex motifs) gives the total.  The sum is carried out in
Python integers (exact beyond 2^64) after gathering the vectors.
"""
from __future__ import annotations

import numpy as np


def heaviest_first(weights: np.ndarray) -> np.ndarray:
    """Vertex ids ordered by weight descending (ties by id)."""
    w = np.asarray(weights)
    return np.lexsort((np.arange(w.shape[0]), -w)).astype(np.int32)


def shard_roots(order: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Round-robin slice of a root order: rank r takes positions r, r+world, ...

    Dealing the heaviest-first order round-robin gives every rank a similar
    mix of heavy and light roots."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return np.ascontiguousarray(order[rank::world], dtype=np.int32)


def reduce_counts(counts, group=None) -> list[int]:
    """Exact elementwise sum of every rank's count vector (all ranks get it)."""
    import torch.distributed as dist
    local = [int(x) for x in counts]
    if not dist.is_available() or not dist.is_initialized():
        return local
    gathered: list = [None] * dist.get_world_size(group)
    dist.all_gather_object(gathered, local, group=group)
    return [sum(col) for col in zip(*gathered)]
