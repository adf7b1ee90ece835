"""The near-alpha comparator (tests/_compare.py) on planted differences (CPU).

A difference counts as hard unless it traces back to a flipped near-alpha
test: the flipped pair itself, or a pair touching an endpoint of it or a
neighbour of such an endpoint.  A near-alpha test that both sides decide
alike excuses nothing.
"""
import numpy as np

from _compare import compare


class _Ref:
    def __init__(self, adj, sepsets, near):
        self.adj = adj
        self.sepsets = sepsets
        self.near = near


def _graph(n, edges):
    adj = np.zeros((n, n), dtype=np.uint8)
    for i, j in edges:
        adj[i, j] = adj[j, i] = 1
    sep = {(i, j): () for i in range(n) for j in range(i + 1, n) if not adj[i, j]}
    return adj, sep


def test_identical_results_have_no_difference():
    adj, sep = _graph(6, [(0, 1), (1, 2), (3, 4)])
    ref = _Ref(adj.copy(), dict(sep), [(0, 1, 0, 0.05)])
    assert compare(adj, sep, ref) == ([], [], [])


def test_difference_without_near_test_is_hard():
    adj, sep = _graph(6, [(0, 1), (1, 2), (3, 4)])
    ref = _Ref(adj.copy(), dict(sep), [])
    g_adj, g_sep = adj.copy(), dict(sep)
    g_sep[(0, 2)] = (1,)                      # a different separating set
    hard, excused, cascade = compare(g_adj, g_sep, ref)
    assert [h[:2] for h in hard] == [(0, 2)] and not excused and not cascade


def test_unflipped_near_test_excuses_nothing():
    adj, sep = _graph(6, [(0, 1), (1, 2), (3, 4)])
    ref = _Ref(adj.copy(), dict(sep), [(0, 1, 0, 0.0500004)])
    g_adj, _ = _graph(6, [(0, 1), (1, 2)])    # (3, 4) removed on one side only
    g_sep = dict(sep)
    g_sep[(3, 4)] = ()
    hard, excused, cascade = compare(g_adj, g_sep, ref)
    assert [h[:2] for h in hard] == [(3, 4)] and not excused and not cascade


def test_flipped_near_test_excuses_its_neighbourhood_only():
    # oracle: path 0-1-2-3 and edge 4-5; the near test of (1, 2) flips on the GPU
    adj, sep = _graph(7, [(0, 1), (1, 2), (2, 3), (4, 5)])
    ref = _Ref(adj.copy(), dict(sep), [(1, 2, 1, 0.049999)])
    g_adj, _ = _graph(7, [(0, 1), (2, 3), (4, 5), (0, 3)])
    g_sep = {k: () for k in sep}
    g_sep.pop((0, 3))
    g_sep[(1, 2)] = (0,)
    g_adj[4, 5] = g_adj[5, 4] = 0             # far from the flip: must stay hard
    g_sep[(4, 5)] = ()
    hard, excused, cascade = compare(g_adj, g_sep, ref)
    assert [e[:2] for e in excused] == [(1, 2)]
    assert [c[:2] for c in cascade] == [(0, 3)]   # 0 is a neighbour of the flipped endpoint 1
    assert [h[:2] for h in hard] == [(4, 5)]
