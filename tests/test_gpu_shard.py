"""fbn_learn_skeleton_sharded on the GPU.

Several processes, one GPU each, learn one skeleton (Section IV-A's
edge-level partition across devices); every process must end with the
oracle's adjacency and separating sets.  This pool gives one GPU per run, so
the processes are emulated by host threads on one GPU, each with its own
handle and stream: they meet only on the host, in the exchange between
depths (no kernel waits on another).  Also: one process owning every edge,
and records that do not describe the shared graph are refused.
"""
import threading

import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare
from paper_2212_04259_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


class _Exchange:
    """The all-gather of the removal records between host threads."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=300)
        self.slots = [None] * world

    def fn(self, rank):
        def exchange(depth, local):
            self.slots[rank] = np.asarray(local, dtype=np.int64).reshape(-1, 3)
            self.bar.wait()
            every = np.concatenate(self.slots)
            self.bar.wait()   # every thread has its copy before the next depth's records arrive
            return every
        return exchange


@pytest.mark.parametrize("name,world", [("small", 1), ("small", 2), ("mid", 2), ("mid", 3)])
def test_sharded_skeleton_matches_oracle(F, name, world):
    import torch
    data, ar, alpha, md, _ = bnsynth.workload(name)
    ref = oracle.pc_stable(data, ar, alpha, md)
    ex = _Exchange(world)
    results, errors = [None] * world, []

    def run(rank):
        try:
            h = F.fbn_create(data, ar, device=0)
            st = torch.cuda.Stream()   # kept alive while the handle runs on it
            F.fbn_set_stream(h, st)
            adj = F.fbn_learn_skeleton_sharded(h, alpha, md, lambda d, a: shard.owned_edges(a, d, rank, world),
                                               ex.fn(rank))
            results[rank] = (adj, F.fbn_export_sepsets(h), F.fbn_get_stats(h))
        except Exception as e:   # pragma: no cover - reported below
            errors.append(e)
            ex.bar.abort()
    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    tests = [0] * len(ref.tests)
    for adj, seps, st in results:
        hard, excused, cascade = compare(adj, seps, ref)
        assert not hard and not excused and not cascade, hard[:3]
        for d, t in enumerate(st["tests_oracle"][: len(tests)]):
            tests[d] += t
    assert tests == ref.tests   # the shares' sequential tests add up to the oracle's


def test_sharded_rejects_records_of_no_edge(F):
    data, ar, alpha, md, _ = bnsynth.workload("small")
    h = F.fbn_create(data, ar)
    with pytest.raises(F.FbnError) as e:
        F.fbn_learn_skeleton_sharded(h, alpha, md, lambda d, a: np.triu(a, 1),
                                     lambda d, local: np.array([[0, 0, 0]], dtype=np.int64))   # i == j: no edge
    assert e.value.code == -1
    # the handle is usable afterwards
    adj = F.fbn_learn_skeleton(h, alpha, md)
    assert np.array_equal(adj, oracle.pc_stable(data, ar, alpha, md).adj)
