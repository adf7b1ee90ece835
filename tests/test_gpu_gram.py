"""Depth 0 on the tensor cores: the one-hot Gram against the oracle.

Every depth-0 contingency table is a block of the Gram matrix of the one-hot
sample matrix.  The counts must be bit-exact, including cells far above 2^14
(the accumulation is flushed to INT32 every 8192 samples) and sample counts
that are not multiples of the 128-sample stage or the 8192-sample chunk.
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


def _offsets(ar):
    return np.concatenate([[0], np.cumsum(ar.astype(np.int64))[:-1]])


def _check_blocks(F, data, ar, pairs):
    h = F.fbn_create(data, ar, depth0="gram")
    G = F.fbn_pairwise_counts(h)
    off = _offsets(ar)
    M = int(ar.astype(np.int64).sum())
    assert G.shape == (M, M) and np.array_equal(G, G.T)
    for i, j in pairs:
        blk = G[off[i]:off[i] + ar[i], off[j]:off[j] + ar[j]].ravel()
        assert np.array_equal(blk, oracle.ci_table(data, ar, int(i), int(j))), (i, j)
    for i in range(len(ar)):   # diagonal blocks: marginal counts on the diagonal
        blk = G[off[i]:off[i] + ar[i], off[i]:off[i] + ar[i]]
        ref = np.bincount(data[i], minlength=int(ar[i]))
        assert np.array_equal(np.diag(blk), ref) and blk.sum() == data.shape[1]
    return G


@pytest.mark.parametrize("N", [1, 127, 129, 8191, 8193, 20011])
def test_pairwise_counts_ragged(F, N):
    rng = np.random.default_rng(N)
    ar = rng.integers(2, 6, 40).astype(np.uint8)
    data = np.stack([rng.integers(0, r, N) for r in ar]).astype(np.uint8)
    pairs = [(i, j) for i in range(40) for j in range(i + 1, 40)]
    _check_blocks(F, data, ar, pairs)


def test_pairwise_counts_many_tiles(F):
    d, a, *_ = bnsynth.workload("mid")
    rng = np.random.default_rng(5)
    ar = rng.integers(2, 6, 300).astype(np.uint8)
    data = np.stack([rng.integers(0, r, 50000) for r in ar]).astype(np.uint8)
    pairs = {(int(i), int(j)) for i, j in rng.integers(0, 300, size=(400, 2)) if i < j}
    pairs |= {(0, 299), (0, 1), (298, 299), (37, 38), (127, 128)}
    _check_blocks(F, data, ar, sorted(pairs))


def test_pairwise_counts_large_cells_exact(F):
    # constant and nearly constant variables: cells of 200,003 and ~190,000,
    # far above what a 14-bit accumulation could hold without flushing
    N = 200003
    rng = np.random.default_rng(9)
    ar = np.array([2, 3, 2, 5, 4, 2], dtype=np.uint8)
    data = np.stack([np.zeros(N, np.int64), np.zeros(N, np.int64),
                     (rng.random(N) < 0.05).astype(np.int64), rng.integers(0, 5, N),
                     rng.integers(0, 4, N), (rng.random(N) < 0.5).astype(np.int64)]).astype(np.uint8)
    G = _check_blocks(F, data, ar, [(i, j) for i in range(6) for j in range(i + 1, 6)])
    assert G[0, 2] == N


def test_depth0_gram_skeleton_matches_oracle(F):
    data, ar, _ = bnsynth.make_dataset(4242, 160, 200, 3, (2, 3, 4, 5), 0.7, 20000)
    ref = oracle.pc_stable(data, ar, 0.05, 1)
    for mode in ("gram", "hist"):
        h = F.fbn_create(data, ar, depth0=mode)
        adj = F.fbn_learn_skeleton(h, 0.05, 1)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard, (mode, hard[:5])
        st = F.fbn_get_stats(h)
        if not ref.near:
            assert st["tests_oracle"] == ref.tests and st["tests"][0] == ref.tests[0]


def test_batched_gram_skeletons_match_oracle(F):
    # a batch large enough to run depth 0 on the tensor cores, problems of
    # different sizes and sample counts
    probs = bnsynth.batched_workload(5, first=10, n_range=(60, 140), samples_range=(3000, 12000))
    hs = [F.fbn_create(d, a, depth0="gram") for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, 1)
    st = F.fbn_get_stats(hs[0])
    assert st["gram_ms"] > 0
    for (d, a, _), h, adj in zip(probs, hs, adjs):
        ref = oracle.pc_stable(d, a, 0.05, 1)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard
    # the same problems one at a time give the same counts
    for (d, a, _), h in zip(probs[:2], hs[:2]):
        G = F.fbn_pairwise_counts(h)
        off = _offsets(a)
        for i, j in [(0, 1), (2, len(a) - 1)]:
            blk = G[off[i]:off[i] + a[i], off[j]:off[j] + a[j]].ravel()
            assert np.array_equal(blk, oracle.ci_table(d, a, i, j))


def test_gram_wait_timeout_is_reported_and_recoverable(F):
    # every bounded wait of the Gram pipeline gives up at once: the kernel
    # issues no copy, releases its tensor memory and reports FBN_ETIMEOUT;
    # the context stays usable
    data, ar, _ = bnsynth.make_dataset(77, 150, 180, 3, (2, 3, 4, 5), 1.0, 9000)
    h = F.fbn_create(data, ar, depth0="gram", wait_limit=-1)
    with pytest.raises(F.FbnError) as e:
        F.fbn_learn_skeleton(h, 0.05, 0)
    assert e.value.code == -6
    h2 = F.fbn_create(data, ar, depth0="gram")
    adj = F.fbn_learn_skeleton(h2, 0.05, 0)
    ref = oracle.pc_stable(data, ar, 0.05, 0)
    assert np.array_equal(adj, ref.adj)
