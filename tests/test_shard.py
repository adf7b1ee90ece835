"""The sharded skeleton's host logic on CPU (paper_2212_04259_gb300.shard).

Several processes learn one skeleton: per depth each tests a weight-balanced
share of the edges (Section IV-A's edge-level partition across devices) and
one all-gather of (i, j, rank) removal records gives every process every
removal.  Here the partition and the all-gather run for real -- two gloo
processes -- and each process's share is tested by a stand-in built from the
oracle's primitives (the sequential tests of Algorithm 1 with the grouping of
Section IV-C, on the CPU); the skeleton and separating sets every process
ends with must equal the sequential oracle's.  The GPU side of the same loop
is tests/test_gpu_shard.py.
"""
import itertools
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bnsynth
import oracle
from paper_2212_04259_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("depth", [0, 1, 2])
def test_owned_edges_partition_the_edges(world, depth):
    rng = np.random.default_rng(world * 10 + depth)
    n = 30
    a = (rng.random((n, n)) < 0.3).astype(np.uint8)
    a = np.triu(a, 1)
    a = a | a.T
    masks = [shard.owned_edges(a, depth, r, world) for r in range(world)]
    total = sum(m.astype(int) for m in masks)
    assert np.array_equal(total, np.triu(a, 1).astype(int))          # every edge once, upper triangle only
    iu, ju, w = shard.edge_weights(a, depth)
    W = w.sum()
    for m in masks:                                                  # balanced within one edge's weight
        share = w[m[iu, ju] == 1].sum()
        assert abs(share - W / world) <= w.max() + 1e-9


def _sharded_oracle(data, ar, alpha, max_depth, rank, world, exchange):
    """The loop of fbn_learn_skeleton_sharded with the oracle testing this
    process's share: returns (adjacency, separating sets)."""
    n = len(ar)
    adj = np.ones((n, n), dtype=np.uint8) - np.eye(n, dtype=np.uint8)
    seps = {}
    d = 0
    while max_depth < 0 or d <= max_depth:
        deg = adj.sum(axis=1)
        if not any(adj[i, j] and max(deg[i], deg[j]) - 1 >= d for i in range(n) for j in range(i + 1, n)):
            break
        nbrs = [list(np.flatnonzero(adj[v])) for v in range(n)]   # the depth's snapshot
        own = shard.owned_edges(adj, d, rank, world)

        def sets(i, j):   # the edge's conditioning sets in rank order
            for a, b in ((i, j), (j, i)):
                cand = [u for u in nbrs[a] if u != b]
                for c in itertools.combinations(cand, d):
                    yield list(c)
        local = []
        for i, j in zip(*np.nonzero(np.triu(own, 1))):
            for r, S in enumerate(sets(int(i), int(j))):
                if oracle.ci_test(data, ar, int(i), int(j), S)[2] > alpha:
                    local.append((int(i), int(j), r))
                    break
        every = exchange(d, np.array(local, dtype=np.int64).reshape(-1, 3))
        for i, j, r in every.tolist():
            seps[(i, j)] = tuple(next(itertools.islice(sets(i, j), r, None)))
        for i, j, _ in every.tolist():
            adj[i, j] = adj[j, i] = 0
        d += 1
    return adj, seps


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data, ar, alpha, md, _ = bnsynth.workload("small", n_samples=3000)
        adj, seps = _sharded_oracle(data, ar, alpha, md, rank, world, shard.allgather_exchange())
        out.put((rank, adj.tolist(), sorted(seps.items())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_processes_learn_the_oracle_skeleton():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    data, ar, alpha, md, _ = bnsynth.workload("small", n_samples=3000)
    ref = oracle.pc_stable(data, ar, alpha, md)
    assert not ref.near
    for _, adj, seps in res:
        assert np.array_equal(np.array(adj, dtype=np.uint8), ref.adj)
        assert dict(seps) == ref.sepsets
