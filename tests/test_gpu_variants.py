"""CI-test variants on the GPU against the oracle: Pearson's X^2 and the
observed-table degrees of freedom, through explicit tests, every depth-0 and
d >= 1 decision path (histogram pool, tensor-core Gram, edge-level form,
sample-split tests) and batches."""
import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu
VARIANTS = [("x2", "fixed"), ("g2", "adjusted"), ("x2", "adjusted")]


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


@pytest.mark.parametrize("stat,mode", VARIANTS)
def test_explicit_tests_match_oracle(F, stat, mode):
    data, ar, *_ = bnsynth.workload("small")
    # a constant-free variable and one with a never-seen level, for the adjusted df
    rng = np.random.default_rng(7)
    extra = np.stack([np.zeros(data.shape[1], np.uint8), (rng.random(data.shape[1]) < 0.3).astype(np.uint8)])
    data = np.concatenate([data, extra])
    ar = np.concatenate([ar, np.array([3, 4], np.uint8)])
    h = F.fbn_create(data, ar, statistic=stat, df=mode)
    n = data.shape[0]
    for x, y, S in [(0, 1, []), (2, 5, [7]), (3, 4, [1, 9]), (n - 2, 0, []), (n - 1, 2, [n - 2]), (5, 6, [8, 10, 12])]:
        st, df, p = F.fbn_ci_test(h, x, y, S)
        rst, rdf, rp = oracle.ci_test(data, ar, x, y, S, stat=stat, df_mode=mode)
        assert df == rdf and st == pytest.approx(rst, rel=1e-6, abs=1e-12) and abs(p - rp) <= 1e-9, (x, y, S)


@pytest.mark.parametrize("opt", [dict(), dict(form="plain"), dict(depth0="gram"), dict(group_size=4)])
@pytest.mark.parametrize("stat,mode", VARIANTS)
@pytest.mark.parametrize("name", ["small", "mid"])
def test_skeleton_parity(F, name, stat, mode, opt):
    data, ar, alpha, md, _ = bnsynth.workload(name)
    ref = oracle.pc_stable(data, ar, alpha, md, stat=stat, df_mode=mode)
    h = F.fbn_create(data, ar, statistic=stat, df=mode, **opt)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard, hard[:5]
    if not ref.near:
        assert F.fbn_get_stats(h)["tests_oracle"] == ref.tests


@pytest.mark.parametrize("stat,mode", VARIANTS)
def test_batch_parity(F, stat, mode):
    probs = bnsynth.batched_workload(6, first=40, n_range=(20, 60), samples_range=(2000, 20000))
    hs = [F.fbn_create(d, a, statistic=stat, df=mode) for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    for (d, a, _), h, adj in zip(probs, hs, adjs):
        ref = oracle.pc_stable(d, a, 0.05, -1, stat=stat, df_mode=mode)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard, hard[:3]


def test_no_degree_of_freedom_removes_the_edge(F):
    rng = np.random.default_rng(2)
    N = 3000
    a = rng.integers(0, 3, N).astype(np.uint8)
    data = np.stack([a, np.zeros(N, np.uint8), a])           # variable 1 constant
    ar = np.array([3, 2, 3], np.uint8)
    for depth0 in ("hist", "gram"):
        h = F.fbn_create(data, ar, df="adjusted", depth0=depth0)
        adj = F.fbn_learn_skeleton(h, 0.05, -1)
        assert not adj[0, 1] and not adj[1, 2] and adj[0, 2], depth0
        assert F.fbn_get_sepset(h, 0, 1) == ()


def test_tensor_depth1_takes_only_the_default_test(F):
    data, ar, *_ = bnsynth.workload("small")
    with pytest.raises(F.FbnError) as e:
        F.fbn_create(data, ar, depth1="tensor", statistic="x2")
    assert e.value.code == -1
