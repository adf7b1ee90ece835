"""Skeleton comparison with the near-alpha rule.

Adjacency and separating sets must be identical to the oracle's, except where
a difference traces back to a test whose oracle p-value lies within the
tolerance of alpha (the oracle logs those tests as ``ref.near``).

A near-alpha pair whose result differs between the two is "flipped".  Its
flip changes the next snapshot only at its two endpoints: the neighbour lists
of those endpoints differ, so every later test of an edge at either endpoint
draws its conditioning sets from a different list, and a removal that
follows from such a test changes the lists of its own endpoints.  A
difference is therefore excused only if

* it is a flipped near-alpha pair itself (``excused``), or
* one of its endpoints is an endpoint of a flipped near-alpha pair, or is a
  neighbour of such an endpoint in either final graph (``cascade``).

Every other difference is ``hard``.  A near-alpha pair that both sides decide
alike excuses nothing, so with no flip every difference is hard.
"""
import numpy as np


def _differs(adj_gpu, sep_gpu, ref, i, j):
    return int(adj_gpu[i, j]) != int(ref.adj[i, j]) or sep_gpu.get((i, j)) != ref.sepsets.get((i, j))


def compare(adj_gpu, sep_gpu, ref):
    """Return (hard, excused, cascade): lists of (i, j, (gpu_adj, oracle_adj, gpu_sep, oracle_sep))."""
    adj_gpu = np.asarray(adj_gpu)
    n = ref.adj.shape[0]
    flipped = {(i, j) for (i, j, _, _) in ref.near if _differs(adj_gpu, sep_gpu, ref, i, j)}
    ends = {v for ij in flipped for v in ij}
    touched = set(ends)
    for v in ends:   # neighbours of a flipped endpoint in either final graph
        touched.update(np.flatnonzero(adj_gpu[v]).tolist())
        touched.update(np.flatnonzero(ref.adj[v]).tolist())
    hard, excused, cascade = [], [], []
    rows, cols = np.nonzero(np.triu(adj_gpu != ref.adj, 1))
    cand = set(zip(rows.tolist(), cols.tolist()))
    cand.update(k for k in set(sep_gpu) | set(ref.sepsets) if sep_gpu.get(k) != ref.sepsets.get(k))
    for (i, j) in sorted(cand):
        item = (i, j, (int(adj_gpu[i, j]), int(ref.adj[i, j]), sep_gpu.get((i, j)), ref.sepsets.get((i, j))))
        if (i, j) in flipped:
            excused.append(item)
        elif i in touched or j in touched:
            cascade.append(item)
        else:
            hard.append(item)
    assert all(0 <= i < j < n for i, j, _ in hard + excused + cascade)
    return hard, excused, cascade
