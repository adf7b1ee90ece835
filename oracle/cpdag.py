"""Oracle of the PC-stable algorithm's second and third steps (Section II-C):
v-structures from the separating sets, then Meek's orientation rules, giving
the completed partially directed graph (CPDAG) of the learned skeleton.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain Python over the
adjacency matrix and the separating sets of ``pc_stable``; the GPU library
has its own implementation and the two share no code.

Encoding of the result M (uint8 [n][n]): M[a][b] = 1 and M[b][a] = 0 for a
directed edge a -> b; M[a][b] = M[b][a] = 1 for an undirected edge; 0 and 0
for no edge.

Readings (the paper states the rules, not their conflict handling):

* v-structure (step 2): for every unshielded triple a - k - b (a < b not
  adjacent, both adjacent to k), k not in SepSet(a, b) puts arrowheads on
  a -> k and b -> k.  All triples are judged on the skeleton alone, so the
  marks do not depend on the order of the triples; an edge that receives
  arrowheads at both ends is left undirected.
* Meek rules R1-R3 (step 3; R4 is needed only with background knowledge),
  applied in rounds: each round collects every orientation any rule implies
  on the current graph, drops the edges that would be oriented both ways,
  applies the rest, and the rounds stop when nothing changes.
    R1  a -> b, b - c, a and c not adjacent             =>  b -> c
    R2  b -> a -> c, b - c                               =>  b -> c
    R3  b - c1 -> c, b - c2 -> c, c1 and c2 not adjacent, b - c  =>  b -> c
"""
from __future__ import annotations

import numpy as np


def _vstructure_marks(adj, sepsets):
    """Arrowhead marks (a, k) for a -> k from the unshielded colliders."""
    n = adj.shape[0]
    marks = set()
    for k in range(n):
        nbrs = [v for v in range(n) if adj[k, v]]
        for x in range(len(nbrs)):
            for y in range(x + 1, len(nbrs)):
                a, b = nbrs[x], nbrs[y]          # a < b (neighbours ascending)
                if adj[a, b]:
                    continue                     # shielded
                if k not in sepsets[(a, b)]:
                    marks.add((a, k))
                    marks.add((b, k))
    return marks


def orient_cpdag(adj, sepsets):
    """CPDAG of a skeleton (uint8 [n][n], symmetric) with its separating sets
    ({(i, j): tuple} for every non-adjacent i < j), as M above."""
    adj = np.asarray(adj, dtype=np.uint8)
    n = adj.shape[0]
    marks = _vstructure_marks(adj, sepsets)
    # directed[a][b] = 1 for a -> b; an edge is undirected when neither is set
    directed = np.zeros((n, n), dtype=np.uint8)
    for a, b in marks:
        if (b, a) not in marks:
            directed[a, b] = 1

    def undirected(a, b):
        return adj[a, b] and not directed[a, b] and not directed[b, a]

    nbrs = [[v for v in range(n) if adj[u, v]] for u in range(n)]
    while True:
        found = set()
        for b in range(n):
            for c in nbrs[b]:
                if not undirected(b, c):
                    continue
                # R1: some a -> b with a, c not adjacent
                r1 = any(directed[a, b] and not adj[a, c] and a != c for a in nbrs[b])
                # R2: some a with b -> a -> c
                r2 = any(directed[b, a] and directed[a, c] for a in nbrs[b])
                # R3: two non-adjacent c1, c2 with b - c1 -> c and b - c2 -> c
                mids = [m for m in nbrs[b] if undirected(b, m) and directed[m, c]]
                r3 = any(not adj[mids[x], mids[y]] for x in range(len(mids)) for y in range(x + 1, len(mids)))
                if r1 or r2 or r3:
                    found.add((b, c))
        new = [(b, c) for (b, c) in found if (c, b) not in found]
        if not new:
            break
        for b, c in new:
            directed[b, c] = 1
    out = np.zeros((n, n), dtype=np.uint8)
    for a in range(n):
        for b in range(n):
            if adj[a, b] and not directed[b, a]:
                out[a, b] = 1
    return out
