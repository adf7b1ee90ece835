"""The device-driven depth loop of Algorithm 1 against the oracle: its bounds
around the depths launched directly (depth 0 on the one-hot Gram, depth 1 on
the neighbourhood product, the edge-level form), repeated calls on one handle
with a changing alpha and maximum depth (the loop graph is captured again and
the critical values refilled), the same kernels driven depth by depth from
the host, and the per-depth statistics the loop records on the device."""
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
    hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard, hard[:5]
    st = F.fbn_get_stats(h)
    assert st["depths"] == len(ref.tests)
    if not ref.near:
        assert st["tests_oracle"] == ref.tests
        assert st["removed"] == ref.removed
    return st


@pytest.mark.parametrize("opt", [dict(), dict(depth0="gram"), dict(depth1="tensor"),
                                 dict(depth0="gram", depth1="tensor"), dict(form="plain"), dict(loop="host"),
                                 dict(loop="host", depth0="gram", depth1="tensor")])
@pytest.mark.parametrize("md", [0, 1, 2, -1])
def test_loop_bounds(F, opt, md):
    data, ar, alpha, _, _ = bnsynth.workload("small")
    ref = oracle.pc_stable(data, ar, alpha, md)
    h = F.fbn_create(data, ar, **opt)
    _check(F, h, F.fbn_learn_skeleton(h, alpha, md), ref)


def test_alpha_and_depth_changes_on_one_handle(F):
    data, ar, _, _, _ = bnsynth.workload("mid")
    h = F.fbn_create(data, ar)
    for alpha, md in [(0.05, -1), (0.01, -1), (0.05, 2), (0.2, -1), (0.05, 0), (0.05, -1)]:
        ref = oracle.pc_stable(data, ar, alpha, md)
        _check(F, h, F.fbn_learn_skeleton(h, alpha, md), ref)


@pytest.mark.parametrize("loop", ["device", "host"])
def test_depth_statistics(F, loop):
    data, ar, alpha, md, _ = bnsynth.workload("mid")
    ref = oracle.pc_stable(data, ar, alpha, md)
    h = F.fbn_create(data, ar, depth0="hist", loop=loop)
    st = _check(F, h, F.fbn_learn_skeleton(h, alpha, md), ref)
    assert st["depths"] >= 3 and st["launches"] > 0
    for d in range(st["depths"]):
        # the depth window (device clock) holds its test kernels' window
        assert st["ms"][d] > 0 and 0 < st["test_ms"][d] <= st["ms"][d], d
        assert st["tests"][d] >= st["tests_oracle"][d] > 0


def test_batch_export_membership(F):
    """A batch's separating sets are compacted for every pending member at the
    first export; members that left (destroyed, new data, learnt again
    alone) are not touched, and the rest still export their own sets."""
    probs = bnsynth.batched_workload(6, first=0, n_range=(20, 40), samples_range=(2000, 8000))
    hs = [F.fbn_create(d, a) for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    F.fbn_destroy(hs[1])                                  # leaves before any export
    F.fbn_update_data(hs[2], probs[2][0])                 # new data: no sets until it learns again
    with pytest.raises(F.FbnError):
        F.fbn_export_sepsets(hs[2])
    d5, a5, _ = probs[5]
    adj5 = F.fbn_learn_skeleton(hs[5], 0.01, -1)          # learnt again alone, at another alpha
    for p in (4, 0, 3):
        d, a, _ = probs[p]
        hard, _, _ = compare(adjs[p], F.fbn_export_sepsets(hs[p]), oracle.pc_stable(d, a, 0.05, -1))
        assert not hard, (p, hard[:3])
    hard, _, _ = compare(adj5, F.fbn_export_sepsets(hs[5]), oracle.pc_stable(d5, a5, 0.01, -1))
    assert not hard
    for p in (0, 2, 3, 4, 5):
        F.fbn_destroy(hs[p])
