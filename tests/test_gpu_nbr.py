"""Depth 1 on the tensor cores: every table (x, y | z) of a vertex's
neighbourhood from one one-hot product, against the oracle.

The skeleton after depth 1, every separating set and the number of tests the
sequential Algorithm 1 runs (which pins the lowest accepting rank of every
edge) must match the oracle.  Cases cover every arity the kernel takes (up to
8, blocks of 64 rows), sample counts that are not multiples of the 128-sample
stage, the 256-sample raw block or the 8192-sample exact accumulation, and
vertices whose neighbourhood needs several row and column tiles.
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


def _check(F, data, ar, alpha, md, **opt):
    ref = oracle.pc_stable(data, ar, alpha, md)
    h = F.fbn_create(data, ar, **opt)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    hard, excused, cascade = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard, hard[:5]
    st = F.fbn_get_stats(h)
    if not ref.near:
        assert st["tests_oracle"] == ref.tests
        assert st["removed"] == ref.removed
    return ref, st


@pytest.mark.parametrize("N", [129, 1000, 8191, 8193, 20011])
def test_depth1_ragged_samples(F, N):
    data, ar, _ = bnsynth.make_dataset(8100 + N % 97, 60, 90, 3, (2, 3, 4), 0.6, N)
    ref, st = _check(F, data, ar, 0.05, 1, depth1="tensor", depth0="hist")
    if len(ref.tests) > 1:
        assert st["tests"][1] >= st["tests_oracle"][1]


@pytest.mark.parametrize("arities", [(2,), (5,), (2, 8), (6, 7, 8), (2, 3, 4, 5, 6, 7, 8)])
def test_depth1_every_arity(F, arities):
    data, ar, _ = bnsynth.make_dataset(8200 + sum(arities), 50, 80, 3, arities, 0.5, 12000)
    _check(F, data, ar, 0.05, 1, depth1="tensor")


def _star(n_children, r_hub, r_child, N, hub_pos, seed):
    # one hub, many children: after depth 0 every child is adjacent to every
    # other (they share the hub), so neighbourhoods span several tiles
    rng = np.random.default_rng(seed)
    hub = rng.integers(0, r_hub, N)
    kids = []
    for _ in range(n_children):
        noise = rng.random(N) < 0.35
        kids.append(np.where(noise, rng.integers(0, r_child, N), hub % r_child))
    rows = kids[:hub_pos] + [hub] + kids[hub_pos:]
    ar = np.array([r_child] * hub_pos + [r_hub] + [r_child] * (n_children - hub_pos), dtype=np.uint8)
    return np.stack(rows).astype(np.uint8), ar


@pytest.mark.parametrize("n_children,r", [(70, 4), (140, 2), (45, 8)])
def test_depth1_hub_spans_tiles(F, n_children, r):
    data, ar = _star(n_children, r, r, 6000, n_children // 4, n_children * 10 + r)
    ref, _ = _check(F, data, ar, 0.05, 1, depth1="tensor")
    assert sum(ref.removed[1:]) > 0   # the children pairs are separated by the hub


def test_depth1_tensor_and_pool_agree(F):
    data, ar, alpha, md, _ = bnsynth.workload("mid")
    out = {}
    for mode in ("tensor", "pool"):
        h = F.fbn_create(data, ar, depth1=mode)
        adj = F.fbn_learn_skeleton(h, alpha, md)
        out[mode] = (adj, F.fbn_export_sepsets(h), F.fbn_get_stats(h)["tests_oracle"])
    assert np.array_equal(out["tensor"][0], out["pool"][0])
    assert out["tensor"][1] == out["pool"][1]
    assert out["tensor"][2] == out["pool"][2]


def test_depth1_batched(F):
    probs = bnsynth.batched_workload(8, first=30, n_range=(20, 90), samples_range=(1000, 20000))
    hs = [F.fbn_create(d, a, depth1="tensor") for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    for (d, a, _), h, adj in zip(probs, hs, adjs):
        ref = oracle.pc_stable(d, a, 0.05, -1)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard, hard[:3]


def test_depth1_wait_timeout_is_reported_and_recoverable(F):
    # every bounded wait of the depth-1 pipeline gives up at once: no copy is
    # issued, tensor memory is released, FBN_ETIMEOUT is reported, and the
    # context stays usable
    data, ar, _ = bnsynth.make_dataset(91, 40, 60, 3, (2, 3, 4), 0.6, 5000)
    h = F.fbn_create(data, ar, depth0="hist", depth1="tensor", wait_limit=-1)
    with pytest.raises(F.FbnError) as e:
        F.fbn_learn_skeleton(h, 0.05, 1)
    assert e.value.code == -6
    _check(F, data, ar, 0.05, 1, depth1="tensor")
