"""Seeded synthetic discrete Bayesian-network data.

This module only draws inputs: a random DAG, random conditional probability
tables and forward-sampled observations, stored variable-major as uint8.  It
holds none of the structure-learning arithmetic (no counting, no test
statistic, no p-value), so both the CPU oracle and the GPU path may take their
inputs from here.

The joint distribution factorises over the DAG as P(V) = prod_i P(V_i | Pa(V_i))
(Section III-A of the Fast-BNS paper); forward sampling draws each variable in
topological order from the CPT row selected by its parents' values.

Workload recipe (the paper's benchmark networks are not available, so seeded
random DAGs of similar size stand in for them):

* topological order pi = a random permutation of the n variables;
* candidate edges pi[a] -> pi[b] (a < b) are drawn uniformly; a candidate is
  rejected when it duplicates an edge or would push the child's in-degree past
  ``max_indegree``; drawing stops at ``n_edges`` edges;
* arities are i.i.d. uniform over ``arities``;
* every CPT row is Dirichlet(dirichlet * 1_r);
* samples are forward-sampled in topological order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Network", "random_network", "sample", "make_dataset", "WORKLOADS",
           "workload", "batched_workload", "batched_size", "chain", "fork", "collider",
           "SEED_BASE", "BATCH_SEED_BASE"]

SEED_BASE = 2212042590        # workload k (1-based) uses SEED_BASE + k
BATCH_SEED_BASE = 2212042600  # problem p of the batched workload uses BATCH_SEED_BASE + p


@dataclasses.dataclass
class Network:
    n: int
    arities: np.ndarray            # uint8 [n]
    parents: list                  # parents[v] = sorted list of parent ids
    order: np.ndarray              # topological order
    cpts: list                     # cpts[v] = float64 [prod(parent arities), r_v]

    def edges(self):
        return sorted((min(p, v), max(p, v)) for v in range(self.n) for p in self.parents[v])


def random_network(rng: np.random.Generator, n: int, n_edges: int, max_indegree: int,
                   arities, dirichlet: float) -> Network:
    arities = np.asarray(list(arities), dtype=np.int64)
    order = rng.permutation(n)
    max_possible = 0
    for b in range(n):
        max_possible += min(b, max_indegree)
    if n_edges > max_possible:
        raise ValueError(f"{n_edges} edges do not fit {n} nodes at in-degree {max_indegree}")
    parents = [set() for _ in range(n)]
    count = 0
    while count < n_edges:
        a, b = rng.integers(0, n, size=2)
        if a == b:
            continue
        if a > b:
            a, b = b, a
        child, parent = int(order[b]), int(order[a])
        if parent in parents[child] or len(parents[child]) >= max_indegree:
            continue
        parents[child].add(parent)
        count += 1
    ar = rng.choice(arities, size=n).astype(np.uint8)
    cpts = []
    for v in range(n):
        pa = sorted(parents[v])
        rows = int(np.prod([int(ar[p]) for p in pa])) if pa else 1
        cpts.append(rng.dirichlet(np.full(int(ar[v]), dirichlet), size=rows))
    return Network(n=n, arities=ar, parents=[sorted(p) for p in parents],
                   order=order, cpts=cpts)


def sample(rng: np.random.Generator, net: Network, n_samples: int) -> np.ndarray:
    """Forward-sample ``n_samples`` rows; returns uint8 [n][n_samples] (variable-major)."""
    data = np.zeros((net.n, n_samples), dtype=np.uint8)
    for v in net.order:
        v = int(v)
        pa = net.parents[v]
        row = np.zeros(n_samples, dtype=np.int64)
        for p in pa:  # mixed-radix parent configuration, first parent most significant
            row = row * int(net.arities[p]) + data[p].astype(np.int64)
        cum = np.cumsum(net.cpts[v], axis=1)[row]          # [N, r_v]
        u = rng.random(n_samples)
        val = (u[:, None] >= cum[:, :-1]).sum(axis=1)
        data[v] = val.astype(np.uint8)
    return data


def make_dataset(seed: int, n: int, n_edges: int, max_indegree: int, arities,
                 dirichlet: float, n_samples: int):
    rng = np.random.default_rng(seed)
    net = random_network(rng, n, n_edges, max_indegree, arities, dirichlet)
    data = sample(rng, net, n_samples)
    return data, net.arities.copy(), net


# The five workloads.  Sizes follow the paper's benchmark range (tens to ~1000
# variables, 5k-200k samples, alpha 0.05/0.01).
WORKLOADS = {
    "small":  dict(index=1, n=20, n_edges=25, max_indegree=3, arities=(2, 3, 4), dirichlet=1.0,
                   n_samples=5000, alpha=0.05, max_depth=-1),
    "mid":    dict(index=2, n=40, n_edges=50, max_indegree=4, arities=(2, 3, 4), dirichlet=0.5,
                   n_samples=50000, alpha=0.05, max_depth=-1),
    "depth0": dict(index=3, n=1000, n_edges=1500, max_indegree=4, arities=(2, 3, 4, 5),
                   dirichlet=1.0, n_samples=200000, alpha=0.05, max_depth=0),
    "large":  dict(index=4, n=1000, n_edges=1200, max_indegree=4, arities=(2, 3, 4, 5),
                   dirichlet=0.5, n_samples=100000, alpha=0.01, max_depth=4),
}


def workload(name: str, n_samples: int | None = None):
    """Return (data uint8 [n][N], arities uint8 [n], alpha, max_depth, net) for a named workload."""
    w = WORKLOADS[name]
    data, ar, net = make_dataset(SEED_BASE + w["index"], w["n"], w["n_edges"], w["max_indegree"],
                                 w["arities"], w["dirichlet"],
                                 w["n_samples"] if n_samples is None else n_samples)
    return data, ar, w["alpha"], w["max_depth"], net


def batched_size(p: int, n_range=(20, 300), samples_range=(1000, 50000)):
    """(n, N) of problem p of the batched workload, without drawing its network or samples."""
    rng = np.random.default_rng(BATCH_SEED_BASE + p)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    lo, hi = math.log(samples_range[0]), math.log(samples_range[1])
    return n, int(round(math.exp(rng.uniform(lo, hi))))


def batched_workload(n_problems: int = 256, first: int = 0, n_range=(20, 300),
                     samples_range=(1000, 50000)):
    """Independent problems of the batched workload: n ~ U{20..300}, N log-uniform in
    [1k, 50k], arities in {2,3,4}, round(1.3 n) edges, in-degree <= 4, Dirichlet(1)."""
    out = []
    for p in range(first, first + n_problems):
        rng = np.random.default_rng(BATCH_SEED_BASE + p)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        lo, hi = math.log(samples_range[0]), math.log(samples_range[1])
        N = int(round(math.exp(rng.uniform(lo, hi))))
        net = random_network(rng, n, int(round(1.3 * n)), 4, (2, 3, 4), 1.0)
        data = sample(rng, net, N)
        out.append((data, net.arities.copy(), net))
    return out


def _tiny(rng, n_samples, spec, strength=0.8):
    """Hand-made faithful DAG on binary variables. spec: list of (child, [parents])."""
    n = 1 + max(max([c] + ps) for c, ps in spec)
    data = np.zeros((n, n_samples), dtype=np.uint8)
    parents = {c: ps for c, ps in spec}
    order, done = [], set()
    while len(order) < n:  # topological order of the hand-made DAG
        for v in range(n):
            if v not in done and all(p in done for p in parents.get(v, [])):
                order.append(v)
                done.add(v)
    for v in order:
        ps = parents.get(v, [])
        if not ps:
            data[v] = (rng.random(n_samples) < 0.5).astype(np.uint8)
        elif len(ps) == 1:
            flip = rng.random(n_samples) >= strength
            data[v] = data[ps[0]] ^ flip.astype(np.uint8)
        else:  # noisy XOR-free OR-like mechanism; both parents matter
            s = data[ps[0]].astype(np.int64) + data[ps[1]].astype(np.int64)
            p1 = np.array([0.1, 0.5, 0.9])[s]
            data[v] = (rng.random(n_samples) < p1).astype(np.uint8)
    return data, np.full(n, 2, dtype=np.uint8)


def chain(n_samples: int = 200000, seed: int = 1):
    """X0 -> X1 -> X2."""
    return _tiny(np.random.default_rng(seed), n_samples, [(1, [0]), (2, [1])])


def fork(n_samples: int = 200000, seed: int = 2):
    """X0 <- X1 -> X2."""
    return _tiny(np.random.default_rng(seed), n_samples, [(0, [1]), (2, [1])])


def collider(n_samples: int = 200000, seed: int = 3):
    """X0 -> X2 <- X1."""
    return _tiny(np.random.default_rng(seed), n_samples, [(2, [0, 1])])
