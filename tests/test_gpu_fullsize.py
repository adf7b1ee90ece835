"""Full-size parity: the workloads at the sizes bench.py times, in its launch
configuration (default options: work pool, group size and ranks per claim
chosen per depth, depth 0 on the tensor-core Gram where the size calls for it).

* large (1000 variables, 100,000 samples, depth <= 4): the whole skeleton and
  every separating set against the oracle's, stored by tests/golden/make_golden.py;
  sampled explicit tests against the oracle.
* depth0 (1000 variables, 200,000 samples): sampled pair decisions and
  bit-exact sampled pair tables against the oracle.
* batched (256 problems): the smallest problems against the oracle in full,
  and on every problem sampled separating sets that must separate.
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
    """The golden file as the oracle's result object."""

    def __init__(self, g):
        n = int(g["n"])
        self.adj = np.zeros((n, n), dtype=np.uint8)
        for i, j in g["edges"]:
            self.adj[i, j] = self.adj[j, i] = 1
        self.sepsets = {(i, j): () for i in range(n) for j in range(i + 1, n) if not self.adj[i, j]}
        off = 0
        for (i, j), L in zip(g["sep_pairs"], g["sep_lens"]):
            self.sepsets[(int(i), int(j))] = tuple(int(v) for v in g["sep_members"][off:off + L])
            off += L
        self.near = [(int(i), int(j), int(d), float(p)) for (i, j, d), p in zip(g["near"], g["near_p"])]
        self.tests = [int(t) for t in g["tests"]]
        self.removed = [int(t) for t in g["removed"]]


def test_large_skeleton_matches_oracle(F):
    path = os.path.join(GOLDEN, "large_skeleton.npz")
    ref = _Ref(np.load(path))
    data, ar, alpha, md, _ = bnsynth.workload("large")
    h = F.fbn_create(data, ar)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard, hard[:5]
    assert len(excused) + len(cascade) <= 20, (excused[:3], cascade[:3])   # one near-alpha flip stays local
    st = F.fbn_get_stats(h)
    if not ref.near:
        assert st["tests_oracle"] == ref.tests
        assert st["removed"] == ref.removed


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


def test_depth0_sampled_pairs(F):
    data, ar, alpha, md, _ = bnsynth.workload("depth0")
    h = F.fbn_create(data, ar)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    st = F.fbn_get_stats(h)
    n = data.shape[0]
    assert st["gram_ms"] > 0 and st["tests"] == [n * (n - 1) // 2]
    rng = np.random.default_rng(8)
    pairs = {(int(min(a, b)), int(max(a, b))) for a, b in rng.integers(0, n, size=(3000, 2)) if a != b}
    for i, j in sorted(pairs):
        _, _, p = oracle.ci_test(data, ar, i, j)
        if abs(p - alpha) <= 1e-6:
            continue
        assert adj[i, j] == (0 if p > alpha else 1), (i, j, p)
    G = F.fbn_pairwise_counts(h)
    off = np.concatenate([[0], np.cumsum(ar.astype(np.int64))[:-1]])
    for i, j in sorted(pairs)[:200]:
        blk = G[off[i]:off[i] + ar[i], off[j]:off[j] + ar[j]].ravel()
        assert np.array_equal(blk, oracle.ci_table(data, ar, i, j))


def test_batched_full_batch(F):
    probs = bnsynth.batched_workload(256)
    hs = [F.fbn_create(d, a) for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    sizes = sorted(range(len(probs)), key=lambda p: probs[p][0].shape[0] * probs[p][0].shape[1])
    for p in sizes[:5]:   # the smallest problems against the oracle in full
        d, a, _ = probs[p]
        ref = oracle.pc_stable(d, a, 0.05, -1)
        hard, _, _ = compare(adjs[p], F.fbn_export_sepsets(hs[p]), ref)
        assert not hard, (p, hard[:3])
    rng = np.random.default_rng(12)
    for p, ((d, a, _), h, adj) in enumerate(zip(probs, hs, adjs)):
        assert np.array_equal(adj, adj.T) and not adj.diagonal().any()
        seps = F.fbn_export_sepsets(h)
        assert set(seps) == {(i, j) for i in range(len(a)) for j in range(i + 1, len(a)) if not adj[i, j]}
        keys = [k for k, S in seps.items() if len(S) > 0]
        for idx in rng.permutation(len(keys))[:3]:
            (i, j) = keys[idx]
            _, _, pv = oracle.ci_test(d, a, i, j, seps[(i, j)])
            assert pv > 0.05 - 1e-6, (p, i, j, seps[(i, j)], pv)
