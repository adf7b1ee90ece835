"""fbn_update_data_batch: new samples for every handle of a batch in one call.

After the batched update (fresh samples of the same networks, same shapes),
the batch's skeletons must be the oracle's on the new data (the bit planes
are rebuilt too), and a value out of range in any data set must be reported,
naming that data set."""
import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu

PROBLEMS = (27, 152, 209)   # small problems of the batched workload: the oracle runs in seconds


def test_batched_update_then_learn():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as F
    first = [bnsynth.batched_workload(1, first=p)[0] for p in PROBLEMS]
    rng = np.random.default_rng(4)
    new = [bnsynth.sample(rng, net, d.shape[1]) for d, _, net in first]
    hs = [F.fbn_create(d, a) for d, a, _ in first]
    F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    F.fbn_update_data_batch(hs, new)
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    for d, (_, a, _), h, adj in zip(new, first, hs, adjs):
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), oracle.pc_stable(d, a, 0.05, -1))
        assert not hard, hard[:3]
    bad = [d.copy() for d in new]
    bad[1][0, 5] = int(first[1][1][0])          # equal to the arity of variable 0 of data set 1
    with pytest.raises(F.FbnError) as e:
        F.fbn_update_data_batch(hs, bad)
    assert e.value.code == -2 and "data set 1" in str(e.value)
