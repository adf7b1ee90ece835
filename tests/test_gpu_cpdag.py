"""PC steps 2-3 (Section II-C) in the library against the oracle: the CPDAG
of a learned skeleton from fbn_orient_cpdag must equal oracle.orient_cpdag
applied to the oracle's skeleton and separating sets, wherever the two
skeletons agree (which the skeleton parity tests establish)."""
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


def _learn(F, data, ar, alpha, md):
    h = F.fbn_create(data, ar)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    return h, adj


def _expect(n, directed=(), undirected=()):
    m = np.zeros((n, n), dtype=np.uint8)
    for a, b in directed:
        m[a, b] = 1
    for a, b in undirected:
        m[a, b] = m[b, a] = 1
    return m


def test_tiny_dags_orient_as_their_equivalence_class(F):
    cases = [(bnsynth.chain, _expect(3, undirected=[(0, 1), (1, 2)])),
             (bnsynth.fork, _expect(3, undirected=[(0, 1), (1, 2)])),
             (bnsynth.collider, _expect(3, directed=[(0, 2), (1, 2)]))]
    for gen, want in cases:
        data, ar = gen()
        h, _ = _learn(F, data, ar, 0.05, -1)
        assert np.array_equal(F.fbn_orient_cpdag(h), want), gen.__name__


def test_rule2_dag_end_to_end(F):
    # 1 -> 3 <- 2, 3 -> 4, 1 -> 4; node 0 unrelated: R1 orients 3 -> 4, R2 orients 1 -> 4
    data, ar = bnsynth._tiny(np.random.default_rng(21), 200000, [(3, [1, 2]), (4, [3, 1])])
    h, adj = _learn(F, data, ar, 0.01, -1)
    want = _expect(5, directed=[(1, 3), (2, 3), (3, 4), (1, 4)])
    assert np.array_equal(F.fbn_orient_cpdag(h), want)


@pytest.mark.parametrize("name", ["small", "mid"])
def test_workload_cpdag_matches_oracle(F, name):
    data, ar, alpha, md, _ = bnsynth.workload(name)
    ref = oracle.pc_stable(data, ar, alpha, md)
    h, adj = _learn(F, data, ar, alpha, md)
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard
    if excused or cascade:
        pytest.skip("a near-alpha decision differs; the CPDAGs may differ with it")
    assert np.array_equal(F.fbn_orient_cpdag(h), oracle.orient_cpdag(ref.adj, ref.sepsets))


def test_large_cpdag_matches_oracle_on_golden(F):
    g = np.load(os.path.join(GOLDEN, "large_skeleton.npz"))
    n = int(g["n"])
    adj_ref = np.zeros((n, n), dtype=np.uint8)
    for i, j in g["edges"]:
        adj_ref[i, j] = adj_ref[j, i] = 1
    seps = {(i, j): () for i in range(n) for j in range(i + 1, n) if not adj_ref[i, j]}
    off = 0
    for (i, j), L in zip(g["sep_pairs"], g["sep_lens"]):
        seps[(int(i), int(j))] = tuple(int(v) for v in g["sep_members"][off:off + L])
        off += L
    data, ar, alpha, md, _ = bnsynth.workload("large")
    h, adj = _learn(F, data, ar, alpha, md)
    if not (np.array_equal(adj, adj_ref) and F.fbn_export_sepsets(h) == seps):
        pytest.skip("a near-alpha decision differs from the golden skeleton; the CPDAGs may differ with it")
    assert np.array_equal(F.fbn_orient_cpdag(h), oracle.orient_cpdag(adj_ref, seps))


def test_orient_before_learning_is_rejected(F):
    data, ar = bnsynth.chain(1000)
    h = F.fbn_create(data, ar)
    with pytest.raises(F.FbnError) as e:
        F.fbn_orient_cpdag(h)
    assert e.value.code == -1
