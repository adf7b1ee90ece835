"""Skeleton comparison with the near-alpha rule.

Adjacency and separating sets must be identical to the oracle's, except where
a difference is traceable to a test whose oracle p-value lies within the
tolerance of alpha (the oracle logs those tests).  A pair with such a test is
excused; once any near-alpha test exists, a flipped removal changes later
snapshots, so other differences are counted as cascade instead of failed.
With no near-alpha test in the oracle run, every difference is a failure.
"""
import numpy as np


def compare(adj_gpu, sep_gpu, ref):
    """Return (hard, excused, cascade): lists of (i, j, detail)."""
    near = {(i, j) for (i, j, _, _) in ref.near}
    hard, excused, cascade = [], [], []
    n = ref.adj.shape[0]
    adj_gpu = np.asarray(adj_gpu)
    for i in range(n):
        for j in range(i + 1, n):
            a, b = int(adj_gpu[i, j]), int(ref.adj[i, j])
            sg, so = sep_gpu.get((i, j)), ref.sepsets.get((i, j))
            if a == b and sg == so:
                continue
            item = (i, j, (a, b, sg, so))
            if (i, j) in near:
                excused.append(item)
            elif near:
                cascade.append(item)
            else:
                hard.append(item)
    return hard, excused, cascade
