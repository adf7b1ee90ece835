"""Several processes, one GPU each, learning one skeleton together.

The edge-level partition of Section IV-A taken across devices: every process
holds the whole sample store and the same graph; at each depth d the edges
are split into contiguous ranges of the canonical order (i < j, row by row)
with about equal work, an edge weighing the conditioning sets it may test,
C(p_i, d) + C(p_j, d) with p_v = |a(V_v)| - 1 (one marginal test at depth 0);
each process tests its range, and one all-gather per depth of the removal
records (i, j, lowest accepting rank) gives every process every removal,
which it applies to the same snapshot (fbn_learn_skeleton_sharded).  The
arithmetic of the tests is the library's; this module only partitions and
exchanges.
"""
from __future__ import annotations

import math

import numpy as np


def edge_weights(adj: np.ndarray, depth: int):
    """Canonical edges (i < j, row by row) of the graph and their weights."""
    a = np.asarray(adj) != 0
    n = a.shape[0]
    deg = a.sum(axis=1)
    iu, ju = np.nonzero(np.triu(a, 1))
    if depth == 0:
        w = np.ones(len(iu), dtype=np.float64)
    else:
        c = np.array([math.comb(int(max(p, 0)), depth) for p in range(n + 1)], dtype=np.float64)
        w = c[np.maximum(deg[iu] - 1, 0)] + c[np.maximum(deg[ju] - 1, 0)]
    return iu, ju, w


def owned_edges(adj: np.ndarray, depth: int, rank: int, world: int) -> np.ndarray:
    """uint8 [n][n] mask (entries i < j) of the edges process `rank` of `world`
    tests at `depth`: the edges whose weight interval's midpoint, in the
    cumulative weights of the canonical order, falls in the rank's share
    [rank W / world, (rank + 1) W / world) of the total W.  The shares
    partition the edges; each holds about W / world, give or take one edge."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    n = np.asarray(adj).shape[0]
    iu, ju, w = edge_weights(adj, depth)
    mask = np.zeros((n, n), dtype=np.uint8)
    if len(iu) == 0:
        return mask
    cum = np.cumsum(w)
    total = cum[-1]
    mid = cum - w / 2.0
    owner = np.minimum((mid * world / total).astype(np.int64), world - 1) if total > 0 else \
        np.arange(len(iu)) * world // len(iu)
    sel = owner == rank
    mask[iu[sel], ju[sel]] = 1
    return mask


def allgather_exchange(group=None):
    """exchange(depth, local) over torch.distributed: every process's records
    (gloo or NCCL process group; the records travel as Python objects)."""
    import torch.distributed as dist

    def exchange(depth, local):
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, np.asarray(local, dtype=np.int64).tolist(), group=group)
        rows = [r for p in parts for r in p]
        return np.array(rows, dtype=np.int64).reshape(-1, 3)
    return exchange


def learn_skeleton_sharded(h, alpha: float, max_depth: int = -1, group=None, adj_out=None):
    """fbn_learn_skeleton_sharded with the partition above and an all-gather
    over the process group (this process's rank and the group's size)."""
    import torch.distributed as dist

    from .fbn import fbn_learn_skeleton_sharded
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    return fbn_learn_skeleton_sharded(h, alpha, max_depth,
                                      lambda d, adj: owned_edges(adj, d, rank, world),
                                      allgather_exchange(group), adj_out=adj_out)
