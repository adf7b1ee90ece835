"""fbn_autotune: choices by measurement, results unchanged.

The autotuner times the skeleton under each candidate configuration (byte
histograms at 32-256 threads per test, bit planes, depth 0 on the Gram or the
histogram) and keeps per depth the fastest.  Whatever it picks, the skeleton
and separating sets must equal the oracle's; options the caller fixed are
kept; FBN_TUNE_AUTO handles tune on their first call and reuse the result for
the same shape.
"""
import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


def _check(F, h, adj, ref):
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard and not excused and not cascade, hard[:3]


def test_autotune_single_keeps_results(F):
    data, ar, alpha, md, _ = bnsynth.workload("mid")
    ref = oracle.pc_stable(data, ar, alpha, md)
    h = F.fbn_create(data, ar)
    t = F.fbn_autotune([h], alpha, md)
    assert t["depths"] == len(ref.tests) and t["candidates"] >= 5
    assert all(c in ("hist", "bits") for c in t["count"])
    assert all(g in (0, 32, 64, 128, 256) for g in t["group_threads"])
    assert t["ms_fixed"] > 0 and t["ms_tuned"] > 0
    adj = F.fbn_learn_skeleton(h, alpha, md)      # runs under the choices
    _check(F, h, adj, ref)
    assert F.fbn_get_stats(h)["tests_oracle"] == ref.tests


def test_autotune_batch_with_gram_keeps_results(F):
    probs = bnsynth.batched_workload(6, first=20, n_range=(60, 140), samples_range=(3000, 12000))
    hs = [F.fbn_create(d, a) for d, a, _ in probs]
    t = F.fbn_autotune(hs, 0.05, -1)
    assert t["depth0"] in ("gram", "hist")
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    for (d, a, _), h, adj in zip(probs, hs, adjs):
        _check(F, h, adj, oracle.pc_stable(d, a, 0.05, -1))


def test_autotune_respects_fixed_options(F):
    data, ar, alpha, md, _ = bnsynth.workload("small")
    h = F.fbn_create(data, ar, group_threads=64, count="hist")
    t = F.fbn_autotune([h], alpha, md)
    assert t["candidates"] == 3 and set(t["count"]) == {"hist"} and set(t["group_threads"]) == {64}
    _check(F, h, F.fbn_learn_skeleton(h, alpha, md), oracle.pc_stable(data, ar, alpha, md))


def test_tune_auto_handles(F):
    data, ar, alpha, md, _ = bnsynth.workload("small")
    ref = oracle.pc_stable(data, ar, alpha, md)
    for _ in range(2):   # the second handle of the same shape reuses the first one's choices
        h = F.fbn_create(data, ar, tune="auto")
        _check(F, h, F.fbn_learn_skeleton(h, alpha, md), ref)
        assert F.fbn_get_stats(h)["tests_oracle"] == ref.tests
