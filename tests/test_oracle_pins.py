"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own code: closed forms, a library
routine the oracle does not call (scipy's G-test and incomplete gamma, mpmath
at 50 digits), brute force on tiny inputs, counting facts the paper prints,
invariants (sum of counts, symmetry, non-negativity), and structure recovery on
tiny faithful DAGs.  A plausible mistake in the oracle (a dropped term, a
swapped marginal, a wrong df, an off-by-one in the subset order, a wrong
decision rule) fails at least one of them.
"""
import itertools
import json
import math
import os

import mpmath
import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

import bnsynth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
mpmath.mp.dps = 50


# --------------------------------------------------------------------------- counts
def _brute_table(data, ar, x, y, S):
    """Pure-Python loop over samples; layout ((z*rx + x)*ry + y), S[0] most significant."""
    cells = int(ar[x]) * int(ar[y]) * int(np.prod([int(ar[s]) for s in S]) if S else 1)
    t = [0] * cells
    for n in range(data.shape[1]):
        z = 0
        for s in S:
            z = z * int(ar[s]) + int(data[s, n])
        t[(z * int(ar[x]) + int(data[x, n])) * int(ar[y]) + int(data[y, n])] += 1
    return np.array(t, dtype=np.int64)


@pytest.mark.parametrize("S", [(), (2,), (2, 3), (4, 2, 3)])
def test_table_matches_brute_force(S):
    rng = np.random.default_rng(7)
    ar = np.array([2, 3, 4, 2, 3], dtype=np.uint8)
    data = np.stack([rng.integers(0, r, 157) for r in ar]).astype(np.uint8)
    got = oracle.ci_table(data, ar, 0, 1, S)
    assert np.array_equal(got, _brute_table(data, ar, 0, 1, list(S)))
    assert got.sum() == data.shape[1]


def test_table_matches_numpy_ravel():
    # independent index arithmetic: numpy's row-major ravel over (S..., X, Y)
    d, a, *_ = bnsynth.workload("small")
    x, y, S = 3, 11, [5, 0, 17]
    dims = [int(a[s]) for s in S] + [int(a[x]), int(a[y])]
    idx = np.ravel_multi_index([d[s] for s in S] + [d[x], d[y]], dims)
    ref = np.bincount(idx, minlength=int(np.prod(dims)))
    assert np.array_equal(oracle.ci_table(d, a, x, y, S), ref)


# --------------------------------------------------------------------------- G^2
def _g2_mp(t2d):
    """Textbook G^2 of a 2-D table at 50 digits: 2 sum N ln(N / E)."""
    t = [[mpmath.mpf(int(v)) for v in row] for row in t2d]
    R = [sum(r) for r in t]
    Cc = [sum(t[i][j] for i in range(len(t))) for j in range(len(t[0]))]
    n = sum(R)
    g = mpmath.mpf(0)
    for i in range(len(t)):
        for j in range(len(t[0])):
            if t[i][j] > 0:
                g += t[i][j] * mpmath.log(t[i][j] * n / (R[i] * Cc[j]))
    return 2 * g


def test_g2_2x2_closed_form():
    # 2x2 closed form: 2[sum a ln a - sum row ln row - sum col ln col + n ln n]
    for a, b, c, d in [(10, 20, 30, 45), (1, 0, 0, 1), (500, 3, 7, 900), (12, 31, 17, 44)]:
        f = lambda v: mpmath.mpf(v) * mpmath.log(v) if v > 0 else mpmath.mpf(0)
        n = a + b + c + d
        ref = 2 * (f(a) + f(b) + f(c) + f(d) - f(a + b) - f(c + d) - f(a + c) - f(b + d) + f(n))
        got = oracle.g2(np.array([a, b, c, d]), 2, 2)
        assert got == pytest.approx(float(ref), rel=1e-13, abs=1e-13)


def test_g2_exact_independence_is_zero():
    # N_xy = N_x N_y / N exactly -> G^2 = 0
    assert oracle.g2(np.array([10, 20, 30, 60]), 2, 2) == 0.0
    assert oracle.g2(np.array([2, 4, 6, 3, 6, 9]), 2, 3) == 0.0


def test_g2_matches_scipy_gtest():
    rng = np.random.default_rng(3)
    for rx, ry in [(2, 2), (2, 5), (4, 3), (5, 5)]:
        for _ in range(5):
            t = rng.integers(1, 300, size=(rx, ry))
            ref = st.chi2_contingency(t, correction=False, lambda_="log-likelihood").statistic
            assert oracle.g2(t.ravel(), rx, ry) == pytest.approx(ref, rel=1e-11)


def test_g2_near_independence_high_precision():
    # near-independent tables: tiny G^2 that a naive FP evaluation loses
    base = np.array([[4000, 8000, 12000], [6000, 12000, 18000]], dtype=np.int64)
    for bump in [(0, 0), (0, 1), (1, 2)]:
        t = base.copy()
        t[bump] += 1
        t[(1 - bump[0], bump[1])] -= 1
        ref = _g2_mp(t)
        got = oracle.g2(t.ravel(), 2, 3)
        assert got == pytest.approx(float(ref), rel=1e-9)
        assert 0 < got < 1e-3


def test_g2_strata_add_up():
    # a 2x2x2 table is the sum of its two 2x2 strata
    s0, s1 = np.array([30, 12, 7, 41]), np.array([5, 22, 19, 3])
    both = np.concatenate([s0, s1])
    assert oracle.g2(both, 2, 2) == pytest.approx(oracle.g2(s0, 2, 2) + oracle.g2(s1, 2, 2), rel=1e-14)
    ref = _g2_mp(s0.reshape(2, 2)) + _g2_mp(s1.reshape(2, 2))
    assert oracle.g2(both, 2, 2) == pytest.approx(float(ref), rel=1e-13)


def test_g2_empty_strata_and_cells():
    # an empty stratum contributes nothing; zero cells are 0 ln 0 = 0
    t = np.array([0, 0, 0, 0, 9, 0, 4, 0])     # second stratum: column y=1 is empty
    assert oracle.g2(t, 2, 2) == 0.0
    t = np.array([0, 0, 0, 0, 9, 1, 0, 4])
    assert oracle.g2(t, 2, 2) == pytest.approx(float(_g2_mp([[9, 1], [0, 4]])), rel=1e-13)


def test_g2_symmetric_and_nonnegative():
    rng = np.random.default_rng(11)
    for _ in range(50):
        rx, ry, nz = rng.integers(2, 6), rng.integers(2, 6), rng.integers(1, 5)
        t = rng.integers(0, 40, size=(nz, rx, ry))
        g = oracle.g2(t.ravel(), rx, ry)
        gt = oracle.g2(np.transpose(t, (0, 2, 1)).ravel(), ry, rx)
        assert g >= 0.0
        assert g == pytest.approx(gt, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------- df
def test_df_conditional_form():
    ar = np.array([2, 3, 4, 5, 2], dtype=np.uint8)
    assert oracle.df(ar, 0, 1) == 2.0              # (2-1)(3-1)
    assert oracle.df(ar, 1, 2, [3]) == 2 * 3 * 5   # (3-1)(4-1) * 5
    assert oracle.df(ar, 3, 4, [0, 2]) == 4 * 1 * 2 * 4


# --------------------------------------------------------------------------- p value
def test_chisq_sf_closed_forms():
    for x in [0.0, 1e-8, 0.3, 1.0, 3.84, 10.0, 50.0, 700.0]:
        assert oracle.chisq_sf(1, x) == pytest.approx(math.erfc(math.sqrt(x / 2)), rel=1e-13, abs=1e-300)
        assert oracle.chisq_sf(2, x) == pytest.approx(math.exp(-x / 2), rel=1e-13, abs=1e-300)
        # df = 4: e^{-t}(1 + t)
        t = x / 2
        assert oracle.chisq_sf(4, x) == pytest.approx(math.exp(-t) * (1 + t), rel=1e-13, abs=1e-300)


def test_chisq_sf_matches_scipy():
    rng = np.random.default_rng(5)
    for k in list(range(1, 40)) + [63, 100, 255, 1000, 4096]:
        for x in np.concatenate([rng.uniform(0, 3 * k, 8), [k, k + 1.0, 0.5 * k]]):
            ref = sp.chdtrc(k, x)
            assert oracle.chisq_sf(k, x) == pytest.approx(ref, rel=1e-10, abs=1e-13)


def test_chisq_sf_large_df_mpmath():
    # at df ~ 1e4 the log-space terms cancel from ~1e5 down to O(1), so the
    # oracle is good to ~1e-11 absolute there: still 100x inside the 1e-9 target
    for k, x in [(10000, 9800.0), (10000, 10150.0), (30000, 29999.0), (2187, 2100.5)]:
        ref = mpmath.gammainc(mpmath.mpf(k) / 2, mpmath.mpf(x) / 2, regularized=True)
        assert oracle.chisq_sf(k, x) == pytest.approx(float(ref), abs=1e-10)


def test_ci_test_consistent_and_decision():
    d, a, *_ = bnsynth.workload("small")
    for x, y, S in [(0, 1, ()), (2, 7, (4,)), (5, 9, (1, 3))]:
        g, df, p = oracle.ci_test(d, a, x, y, S)
        t = oracle.ci_table(d, a, x, y, S)
        assert g == oracle.g2(t, int(a[x]), int(a[y]))
        assert df == oracle.df(a, x, y, S)
        assert p == oracle.chisq_sf(int(df), g)
        assert 0.0 <= p <= 1.0


# --------------------------------------------------------------------------- subsets
def test_subsets_lexicographic():
    for p in range(0, 13):
        for q in range(0, 6):
            assert oracle.subsets(p, q) == list(itertools.combinations(range(p), q))


def test_subset_counts_printed_in_paper():
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        g = json.load(f)
    for row in g["conditioning_set_counts"]:
        assert len(oracle.subsets(row["p"], row["q"])) == row["count"]


# --------------------------------------------------------------------------- skeleton
def _edges(adj):
    n = adj.shape[0]
    return {(i, j) for i in range(n) for j in range(i + 1, n) if adj[i, j]}


def test_chain_fork_collider_recovery():
    d, a = bnsynth.chain()
    r = oracle.pc_stable(d, a, 0.05)
    assert _edges(r.adj) == {(0, 1), (1, 2)}
    assert r.sepsets == {(0, 2): (1,)}
    d, a = bnsynth.fork()
    r = oracle.pc_stable(d, a, 0.05)
    assert _edges(r.adj) == {(0, 1), (1, 2)}
    assert r.sepsets == {(0, 2): (1,)}
    d, a = bnsynth.collider()
    r = oracle.pc_stable(d, a, 0.05)
    assert _edges(r.adj) == {(0, 2), (1, 2)}
    assert r.sepsets == {(0, 1): ()}


def test_depth0_test_count_and_independent_data():
    # fully independent variables: depth 0 runs n(n-1)/2 tests and (almost) all edges go
    rng = np.random.default_rng(0)
    n = 12
    ar = rng.integers(2, 5, n).astype(np.uint8)
    data = np.stack([rng.integers(0, r, 20000) for r in ar]).astype(np.uint8)
    r = oracle.pc_stable(data, ar, 0.01, max_depth=0)
    assert r.tests[0] == n * (n - 1) // 2
    assert len(r.tests) == 1


def test_adjacency_symmetric_and_sepsets_consistent():
    d, a, alpha, md, _ = bnsynth.workload("small")
    r = oracle.pc_stable(d, a, alpha, md)
    assert np.array_equal(r.adj, r.adj.T) and not r.adj.diagonal().any()
    n = d.shape[0]
    for i in range(n):
        for j in range(i + 1, n):
            assert (r.adj[i, j] == 0) == ((i, j) in r.sepsets)
    # every stored separating set really separates: its test accepts independence
    for (i, j), S in r.sepsets.items():
        _, _, p = oracle.ci_test(d, a, i, j, S)
        assert p > alpha


def test_skeleton_permutation_invariant():
    d, a, alpha, md, _ = bnsynth.workload("small")
    r = oracle.pc_stable(d, a, alpha, md)
    perm = np.random.default_rng(4).permutation(d.shape[0])
    rp = oracle.pc_stable(d[perm], a[perm], alpha, md)
    # variable perm[k] of the original is variable k of the permuted problem
    back = rp.adj[np.ix_(np.argsort(perm), np.argsort(perm))]
    assert np.array_equal(back, r.adj)


def test_max_depth_stops():
    d, a, alpha, _, _ = bnsynth.workload("small")
    full = oracle.pc_stable(d, a, alpha, -1)
    r1 = oracle.pc_stable(d, a, alpha, 1)
    assert len(r1.tests) == 2 and r1.tests == full.tests[:2]
    assert all(len(S) <= 1 for S in r1.sepsets.values())


# ------------------------------------------------------------- brute-force PC-stable
def _py_pc_stable(data, ar, alpha, edge_order_seed=None):
    """Independent tiny PC-stable: numpy counts, per-stratum G^2 in mpmath, scipy p.
    With edge_order_seed, the edges of each depth are tested in a random order
    (every edge reads the same snapshot, as the edge-parallel form does)."""
    n = data.shape[0]
    adj = np.ones((n, n), dtype=bool)
    np.fill_diagonal(adj, False)
    sep = {}

    def test(i, j, S):
        dims = [int(ar[s]) for s in S] + [int(ar[i]), int(ar[j])]
        t = np.bincount(np.ravel_multi_index([data[s] for s in S] + [data[i], data[j]], dims),
                        minlength=int(np.prod(dims))).reshape(-1, int(ar[i]), int(ar[j]))
        g = mpmath.mpf(0)
        for stratum in t:
            if stratum.sum() > 0:
                g += _g2_mp(stratum)
        df = (int(ar[i]) - 1) * (int(ar[j]) - 1) * int(np.prod([int(ar[s]) for s in S]) if S else 1)
        return float(sp.chdtrc(df, float(g)))

    d = 0
    while True:
        a = {v: sorted(np.flatnonzero(adj[v]).tolist()) for v in range(n)}
        if not any(len(a[i]) - 1 >= d for i in range(n) for _ in a[i]):
            break
        rm = []
        pairs = [(i, j) for i in range(n) for j in a[i] if j > i]
        if edge_order_seed is not None:
            order = np.random.default_rng(edge_order_seed + d).permutation(len(pairs))
            pairs = [pairs[k] for k in order]
        for i, j in pairs:
            done = False
            for side in ((i, j), (j, i))[: 1 if d == 0 else 2]:
                cand = [v for v in a[side[0]] if v != side[1]]
                for S in itertools.combinations(cand, d):
                    if test(i, j, list(S)) > alpha:
                        rm.append((i, j))
                        sep[(i, j)] = tuple(S)
                        done = True
                        break
                if done:
                    break
        for i, j in rm:
            adj[i, j] = adj[j, i] = False
        d += 1
    return adj.astype(np.uint8), sep


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_skeleton_matches_brute_force(seed):
    data, ar, _ = bnsynth.make_dataset(1000 + seed, 7, 8, 3, (2, 3), 0.7, 3000)
    adj, sep = _py_pc_stable(data, ar, 0.05)
    r = oracle.pc_stable(data, ar, 0.05)
    if r.near:
        pytest.skip("near-alpha tie in this draw")
    assert np.array_equal(r.adj, adj)
    assert r.sepsets == sep


def test_edge_parallel_form_equals_the_sequential_oracle():
    # PC-stable (Algorithm 1): the edges of a depth read one snapshot, so any
    # order of testing them -- the edge-parallel form -- gives the oracle's result
    data, ar, _ = bnsynth.make_dataset(1010, 7, 8, 3, (2, 3), 0.7, 3000)
    r = oracle.pc_stable(data, ar, 0.05)
    if r.near:
        pytest.skip("near-alpha tie in this draw")
    for order_seed in (11, 12):
        adj, sep = _py_pc_stable(data, ar, 0.05, edge_order_seed=order_seed)
        assert np.array_equal(r.adj, adj) and r.sepsets == sep
