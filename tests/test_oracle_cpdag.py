"""Pins of the oracle's PC steps 2-3 (Section II-C): v-structures from the
separating sets, then Meek's rules R1-R3.

Beyond hand-built cases for each rule, the oracle is checked against a brute
force: for small random DAGs, the CPDAG of the Markov equivalence class is
computed by enumerating every orientation of the skeleton that is acyclic and
has the DAG's v-structures (Verma and Pearl: same skeleton and v-structures
<=> Markov equivalent) and keeping the edges oriented alike in all of them.
The oracle gets the DAG's skeleton and separating sets that d-separate (the
parents of whichever endpoint is not an ancestor of the other); Meek's rules
are complete, so the two must agree exactly.
"""
import itertools

import numpy as np
import pytest

import oracle


def _skeleton(n, edges):
    adj = np.zeros((n, n), dtype=np.uint8)
    for a, b in edges:
        adj[a, b] = adj[b, a] = 1
    return adj


def _expect(n, directed=(), undirected=()):
    m = np.zeros((n, n), dtype=np.uint8)
    for a, b in directed:
        m[a, b] = 1
    for a, b in undirected:
        m[a, b] = m[b, a] = 1
    return m


def _seps(n, adj, given):
    s = {(i, j): () for i in range(n) for j in range(i + 1, n) if not adj[i, j]}
    s.update(given)
    return s


def test_collider_chain_fork():
    adj = _skeleton(3, [(0, 2), (1, 2)])
    got = oracle.orient_cpdag(adj, _seps(3, adj, {(0, 1): ()}))
    assert np.array_equal(got, _expect(3, directed=[(0, 2), (1, 2)]))
    adj = _skeleton(3, [(0, 1), (1, 2)])
    got = oracle.orient_cpdag(adj, _seps(3, adj, {(0, 2): (1,)}))
    assert np.array_equal(got, _expect(3, undirected=[(0, 1), (1, 2)]))


def test_rule1_propagates_away_from_a_collider():
    adj = _skeleton(4, [(0, 2), (1, 2), (2, 3)])
    got = oracle.orient_cpdag(adj, _seps(4, adj, {(0, 1): (), (0, 3): (2,), (1, 3): (2,)}))
    assert np.array_equal(got, _expect(4, directed=[(0, 2), (1, 2), (2, 3)]))


def test_rule2_closes_a_directed_path():
    # 1 -> 3 <- 2 (collider), 3 - 4 by R1 (2 not adjacent to 4), then 1 - 4 by R2
    adj = _skeleton(5, [(1, 3), (2, 3), (3, 4), (1, 4)])
    seps = _seps(5, adj, {(1, 2): (), (2, 4): (1, 3)})
    for v in (0,):
        for u in range(1, 5):
            seps[(v, u)] = ()
    got = oracle.orient_cpdag(adj, seps)
    assert np.array_equal(got, _expect(5, directed=[(1, 3), (2, 3), (3, 4), (1, 4)]))


def test_rule3_two_undirected_paths_into_a_collider():
    a, b, c, d = 0, 1, 2, 3
    adj = _skeleton(4, [(c, b), (d, b), (a, c), (a, d), (a, b)])
    got = oracle.orient_cpdag(adj, _seps(4, adj, {(c, d): (a,)}))
    assert np.array_equal(got, _expect(4, directed=[(c, b), (d, b), (a, b)], undirected=[(a, c), (a, d)]))


def test_conflicting_colliders_leave_the_edge_undirected():
    # 0 - 1 - 2 - 3 with empty separating sets: colliders at 1 and at 2 mark
    # 1 - 2 both ways; R1 would orient it both ways too, so it stays undirected
    adj = _skeleton(4, [(0, 1), (1, 2), (2, 3)])
    got = oracle.orient_cpdag(adj, _seps(4, adj, {}))
    assert np.array_equal(got, _expect(4, directed=[(0, 1), (3, 2)], undirected=[(1, 2)]))


# ---------------------------------------------------------------- brute force
def _descendants(n, parents):
    children = [[] for _ in range(n)]
    for v in range(n):
        for p in parents[v]:
            children[p].append(v)
    out = []
    for v in range(n):
        seen, stack = set(), list(children[v])
        while stack:
            u = stack.pop()
            if u not in seen:
                seen.add(u)
                stack.extend(children[u])
        out.append(seen)
    return out


def _vstructs(n, arcs):
    par = [set() for _ in range(n)]
    for a, b in arcs:
        par[b].add(a)
    adj = set(arcs) | {(b, a) for a, b in arcs}
    return {(min(a, b), k, max(a, b)) for k in range(n) for a in par[k] for b in par[k]
            if a != b and (a, b) not in adj}


def _acyclic(n, arcs):
    par = [set() for _ in range(n)]
    for a, b in arcs:
        par[b].add(a)
    state = [0] * n

    def visit(v):
        state[v] = 1
        for p in par[v]:
            if state[p] == 1 or (state[p] == 0 and not visit(p)):
                return False
        state[v] = 2
        return True

    return all(state[v] == 2 or visit(v) for v in range(n))


def _cpdag_bruteforce(n, arcs):
    edges = sorted({(min(a, b), max(a, b)) for a, b in arcs})
    target = _vstructs(n, arcs)
    members = []
    for bits in itertools.product((0, 1), repeat=len(edges)):
        cand = [(a, b) if f == 0 else (b, a) for (a, b), f in zip(edges, bits)]
        if _acyclic(n, cand) and _vstructs(n, cand) == target:
            members.append(set(cand))
    m = np.zeros((n, n), dtype=np.uint8)
    for a, b in edges:
        if all((a, b) in s for s in members):
            m[a, b] = 1
        elif all((b, a) in s for s in members):
            m[b, a] = 1
        else:
            m[a, b] = m[b, a] = 1
    return m


@pytest.mark.parametrize("seed", range(60))
def test_matches_bruteforce_cpdag_of_random_dags(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(3, 7))
    order = rng.permutation(n)
    arcs = [(int(order[i]), int(order[j])) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.45]
    arcs = arcs[:10]
    parents = [set() for _ in range(n)]
    for a, b in arcs:
        parents[b].add(a)
    desc = _descendants(n, parents)
    adj = _skeleton(n, arcs)
    seps = {}
    for i in range(n):
        for j in range(i + 1, n):
            if adj[i, j]:
                continue
            s = parents[j] if i not in desc[j] else parents[i]
            seps[(i, j)] = tuple(sorted(s))
    assert np.array_equal(oracle.orient_cpdag(adj, seps), _cpdag_bruteforce(n, arcs))
