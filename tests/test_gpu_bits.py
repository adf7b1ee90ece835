"""Bit-plane counting against the oracle.

Tables of tests whose variables all have arity <= 4 (and at most two
conditioning variables) can be counted from two bit planes per variable with
popcounts (count="bits" forces it wherever it fits, count="auto" uses it for
small tables).  Tables must be bit-exact, G^2 within 1e-6 relative and p
within 1e-9 absolute of the oracle, and skeletons and separating sets
identical to the oracle's (the near-alpha rule of tests/_compare.py).
Covered: every value of every arity (minterms 0-3 and the zero padding),
sample counts around the 32-sample word and the 128-sample group, tables
with arities above 4 (counted by the byte histogram instead), explicit tests
(a CTA group) and the work pool at every group size, with sample-split
tests, single problems and a batch.
"""
import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu
G2_REL, P_ABS = 1e-6, 1e-9


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


def _rand(seed, arities, N, skew=False):
    rng = np.random.default_rng(seed)
    rows = []
    for r in arities:
        if skew:   # mostly the top value: the all-ones minterm
            rows.append(np.where(rng.random(N) < 0.7, r - 1, rng.integers(0, r, N)))
        else:
            rows.append(rng.integers(0, r, N))
    return np.stack(rows).astype(np.uint8), np.array(arities, dtype=np.uint8)


@pytest.mark.parametrize("N", [1, 31, 32, 33, 127, 128, 129, 1000, 4097, 65537])
def test_bits_tables_ragged_samples(F, N):
    data, ar = _rand(N, [4, 3, 2, 4, 3], N)
    h = F.fbn_create(data, ar, count="bits")
    for x, y, S in [(0, 1, []), (2, 0, [1]), (3, 4, [0, 2]), (1, 3, [4]), (4, 2, [3, 0])]:
        got = F.fbn_ci_table(h, x, y, S)
        ref = oracle.ci_table(data, ar, x, y, S)
        assert np.array_equal(got[: ref.size], ref), (N, x, y, S)


@pytest.mark.parametrize("skew", [False, True])
def test_bits_tests_match_oracle(F, skew):
    data, ar = _rand(11 + skew, [2, 3, 4, 4, 2, 3, 5, 4], 30011, skew=skew)
    hb = F.fbn_create(data, ar, count="bits")
    hh = F.fbn_create(data, ar, count="hist")
    rng = np.random.default_rng(5)
    for _ in range(60):
        d = int(rng.integers(0, 3))
        v = rng.permutation(len(ar))[: d + 2]
        x, y, S = int(v[0]), int(v[1]), [int(t) for t in v[2:]]
        rg2, rdf, rp = oracle.ci_test(data, ar, x, y, S)
        for h in (hb, hh):
            g2, df, p = F.fbn_ci_test(h, x, y, S)
            assert df == rdf and g2 == pytest.approx(rg2, rel=G2_REL, abs=1e-12) and abs(p - rp) <= P_ABS
        assert np.array_equal(F.fbn_ci_table(hb, x, y, S), oracle.ci_table(data, ar, x, y, S))


def test_bits_constant_and_top_values(F):
    # constant rows (only one minterm occupied), rows at the top value only
    N = 5003
    data = np.stack([np.zeros(N), np.full(N, 3), np.full(N, 1), np.arange(N) % 4, (np.arange(N) // 7) % 3]
                    ).astype(np.uint8)
    ar = np.array([2, 4, 3, 4, 3], dtype=np.uint8)
    h = F.fbn_create(data, ar, count="bits")
    for x, y, S in [(0, 1, []), (1, 3, [4]), (3, 4, [0, 2]), (2, 3, [1])]:
        assert np.array_equal(F.fbn_ci_table(h, x, y, S), oracle.ci_table(data, ar, x, y, S))
        g2, df, p = F.fbn_ci_test(h, x, y, S)
        rg2, rdf, rp = oracle.ci_test(data, ar, x, y, S)
        assert df == rdf and g2 == pytest.approx(rg2, rel=G2_REL, abs=1e-12) and abs(p - rp) <= P_ABS


@pytest.mark.parametrize("gt", [0, 32, 64, 128, 256])
@pytest.mark.parametrize("count", ["auto", "bits"])
def test_bits_skeletons_match_oracle(F, gt, count):
    for name in ("small", "mid"):
        data, ar, alpha, md, _ = bnsynth.workload(name)
        ref = oracle.pc_stable(data, ar, alpha, md)
        h = F.fbn_create(data, ar, group_threads=gt, count=count)
        adj = F.fbn_learn_skeleton(h, alpha, md)
        hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard and not excused and not cascade, (name, gt, count, hard[:3])
        st = F.fbn_get_stats(h)
        assert st["tests_oracle"] == ref.tests and st["removed"] == ref.removed


def test_bits_skeleton_mixed_arities(F):
    # arities up to 5: tests with an arity-5 variable fall back to the histogram
    data, ar, _ = bnsynth.make_dataset(515, 30, 40, 3, (2, 3, 4, 5), 0.7, 20000)
    ref = oracle.pc_stable(data, ar, 0.05, -1)
    for count in ("auto", "bits"):
        h = F.fbn_create(data, ar, count=count)
        adj = F.fbn_learn_skeleton(h, 0.05, -1)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard, (count, hard[:3])


def test_bits_batch_matches_oracle(F):
    probs = bnsynth.batched_workload(8, first=40)
    for count in ("auto", "bits"):
        hs = [F.fbn_create(d, a, count=count) for d, a, _ in probs]
        adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
        for (d, a, _), h, adj in zip(probs, hs, adjs):
            ref = oracle.pc_stable(d, a, 0.05, -1)
            hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
            assert not hard, (count, hard[:3])


def test_bits_update_data_rebuilds_planes(F):
    d1, ar = _rand(1, [3, 4, 2, 4], 9001)
    d2, _ = _rand(2, [3, 4, 2, 4], 9001)
    h = F.fbn_create(d1, ar, count="bits")
    assert np.array_equal(F.fbn_ci_table(h, 0, 1, [2]), oracle.ci_table(d1, ar, 0, 1, [2]))
    F.fbn_update_data(h, d2)
    assert np.array_equal(F.fbn_ci_table(h, 0, 1, [2]), oracle.ci_table(d2, ar, 0, 1, [2]))
    assert np.array_equal(F.fbn_ci_table(h, 3, 1, [0, 2]), oracle.ci_table(d2, ar, 3, 1, [0, 2]))
