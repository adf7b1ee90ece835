"""Full-size parity: the workloads at the sizes bench.py times, in its launch
configuration (default options: work pool, group size and ranks per claim
chosen per depth, depth 0 on the tensor-core Gram where the size calls for it).
The expected values are the oracle's, stored by tests/golden/make_golden.py.

* large (1000 variables, 100,000 samples, depth <= 4): the whole skeleton and
  every separating set against the oracle's; sampled explicit tests.
* depth0 (1000 variables, 200,000 samples): the decision of every one of the
  499,500 pairs; every pair table's margins (full size: each block of the
  one-hot Gram sums, row by row and column by column, to the two variables'
  value counts); sampled pair tables bit-exact against the oracle.
* batched (256 problems): every problem's skeleton and separating sets.

Differences are allowed only where the comparator traces them to a flipped
near-alpha test (tests/_compare.py); with no flip, results must be identical.
"""
import os

import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


class _Ref:
    """One oracle skeleton from a golden record, as the oracle's result object."""

    def __init__(self, n, edges, sep_pairs, sep_lens, sep_members, near, near_p, tests, removed):
        self.adj = np.zeros((n, n), dtype=np.uint8)
        for i, j in edges:
            self.adj[i, j] = self.adj[j, i] = 1
        self.sepsets = {(i, j): () for i in range(n) for j in range(i + 1, n) if not self.adj[i, j]}
        off = 0
        for (i, j), L in zip(sep_pairs.tolist(), sep_lens.tolist()):   # Python ints (stored narrow)
            self.sepsets[(i, j)] = tuple(int(v) for v in sep_members[off:off + L])
            off += L
        self.near = [(int(i), int(j), int(d), float(p)) for (i, j, d), p in zip(near, near_p)]
        self.tests = [int(t) for t in tests]
        self.removed = [int(t) for t in removed]


def _large_ref():
    g = np.load(os.path.join(GOLDEN, "large_skeleton.npz"))
    return _Ref(int(g["n"]), g["edges"], g["sep_pairs"], g["sep_lens"], g["sep_members"], g["near"], g["near_p"],
                g["tests"], g["removed"])


def _batched_refs():
    g = np.load(os.path.join(GOLDEN, "batched_skeletons.npz"))
    refs = []
    for p in range(int(g["n_problems"])):
        part = {f: g[f][g[f + "_off"][p]:g[f + "_off"][p + 1]]
                for f in ("edges", "sep_pairs", "sep_lens", "sep_members", "near", "near_p", "tests", "removed")}
        refs.append(_Ref(int(g["n"][p]), **part))
    return refs


def test_large_skeleton_matches_oracle(F):
    ref = _large_ref()
    data, ar, alpha, md, _ = bnsynth.workload("large")
    h = F.fbn_create(data, ar)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard, hard[:5]
    st = F.fbn_get_stats(h)
    if not excused and not cascade:   # no near-alpha flip: identical, down to the per-depth counts
        assert st["tests_oracle"] == ref.tests
        assert st["removed"] == ref.removed
        assert st["test_samples"] == [t * data.shape[1] for t in ref.tests]


def test_large_sampled_tests(F):
    data, ar, *_ = bnsynth.workload("large")
    h = F.fbn_create(data, ar)
    rng = np.random.default_rng(31)
    for _ in range(40):
        d = int(rng.integers(0, 5))
        v = rng.permutation(data.shape[0])[: d + 2]
        x, y, S = int(v[0]), int(v[1]), [int(t) for t in v[2:]]
        g2, df, p = F.fbn_ci_test(h, x, y, S)
        rg2, rdf, rp = oracle.ci_test(data, ar, x, y, S)
        assert df == rdf and g2 == pytest.approx(rg2, rel=1e-6, abs=1e-12) and abs(p - rp) <= 1e-9


def test_depth0_every_pair(F):
    g = np.load(os.path.join(GOLDEN, "depth0_pairs.npz"))
    data, ar, alpha, md, _ = bnsynth.workload("depth0")
    n, N = data.shape
    h = F.fbn_create(data, ar)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    st = F.fbn_get_stats(h)
    assert st["gram_ms"] > 0 and st["tests"] == [n * (n - 1) // 2]
    kept = np.unpackbits(g["kept_bits"])[: int(g["n_pairs"])].astype(bool)
    iu, ju = np.triu_indices(n, 1)                     # row by row, as the golden file
    got = adj[iu, ju].astype(bool)
    near = {(int(i), int(j)) for i, j in g["near"]}
    diff = [(int(i), int(j)) for i, j in zip(iu[got != kept], ju[got != kept])]
    assert all(d in near for d in diff), [d for d in diff if d not in near][:5]   # depth 0: a flip stays local
    assert np.array_equal(adj, adj.T) and not adj.diagonal().any()
    # every pair table through its margins, at full size
    G = F.fbn_pairwise_counts(h)
    off = np.concatenate([[0], np.cumsum(ar.astype(np.int64))])
    marg = np.concatenate([np.bincount(data[v], minlength=int(ar[v])) for v in range(n)])
    assert np.array_equal(G, G.T)
    for i in range(n):
        rows = G[off[i]:off[i + 1]]                     # blocks (i, j) for every j
        sums = np.add.reduceat(rows, off[:-1], axis=1)  # [r_i][n]: row sums of each block
        assert np.array_equal(sums, np.repeat(marg[off[i]:off[i + 1], None], n, axis=1)), i
    assert np.array_equal(np.diagonal(G), marg)
    # sampled pair tables bit-exact
    rng = np.random.default_rng(8)
    for a, b in rng.integers(0, n, size=(300, 2)):
        if a == b:
            continue
        i, j = int(min(a, b)), int(max(a, b))
        blk = G[off[i]:off[i + 1], off[j]:off[j + 1]].ravel()
        assert np.array_equal(blk, oracle.ci_table(data, ar, i, j))


def test_batched_every_problem(F):
    refs = _batched_refs()
    probs = bnsynth.batched_workload(len(refs))
    hs = [F.fbn_create(d, a) for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    flips = 0
    for p, (ref, h, adj) in enumerate(zip(refs, hs, adjs)):
        hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard, (p, hard[:3])
        flips += len(excused) + len(cascade)
    st = F.fbn_get_stats(hs[0])   # the batch's counters
    if flips == 0:
        depth = max(len(r.tests) for r in refs)
        tests = [sum(r.tests[d] for r in refs if d < len(r.tests)) for d in range(depth)]
        removed = [sum(r.removed[d] for r in refs if d < len(r.removed)) for d in range(depth)]
        samples = [sum(r.tests[d] * probs[p][0].shape[1] for p, r in enumerate(refs) if d < len(r.tests))
                   for d in range(depth)]
        assert st["tests_oracle"] == tests
        assert st["removed"] == removed
        assert st["test_samples"] == samples
