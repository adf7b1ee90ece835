"""Write the oracle's skeletons of the full-size workloads as golden files.

Runs only the CPU oracle (``oracle/``) on the seeded workloads and stores what
the GPU parity tests compare element by element at full size:

* ``large``   (1000 variables, 1200 edges, 100,000 samples, alpha 0.01,
  depth <= 4): the remaining edges, every non-empty separating set (removed
  pairs not listed have the empty set), tests and removals per depth, and
  the tests whose p-value lies within 1e-6 of alpha;
* ``depth0``  (1000 variables, 200,000 samples, depth 0 only): the decision
  of every one of the n(n-1)/2 = 499,500 pairs (the kept pairs as a bit per
  pair of the upper triangle, row by row) and the near-alpha tests;
* ``batched`` (256 independent problems, 20-300 variables, 1k-50k samples,
  alpha 0.05, unbounded depth): for every problem the same record as for
  ``large``, problem after problem, with per-problem offsets.

The oracle is sequential; independent problems (and, for depth0, blocks of
pairs) run in separate processes (spawn) on the host cores.

    python tests/golden/make_golden.py [large|depth0|batched] [--procs P]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bnsynth  # noqa: E402
import oracle   # noqa: E402


def _record(r, n):
    """Edges, non-empty separating sets, per-depth counts and near-alpha tests of one oracle run."""
    edges = np.array([(i, j) for i in range(n) for j in range(i + 1, n) if r.adj[i, j]],
                     dtype=np.int32).reshape(-1, 2)
    nonempty = sorted((k, v) for k, v in r.sepsets.items() if len(v) > 0)
    pairs = np.array([k for k, _ in nonempty], dtype=np.int32).reshape(-1, 2)
    lens = np.array([len(v) for _, v in nonempty], dtype=np.int32)
    members = np.array([m for _, v in nonempty for m in v], dtype=np.int32)
    near = np.array([(i, j, d) for (i, j, d, _) in r.near], dtype=np.int32).reshape(-1, 3)
    near_p = np.array([p for (_, _, _, p) in r.near], dtype=np.float64)
    return dict(edges=edges, sep_pairs=pairs, sep_lens=lens, sep_members=members,
                tests=np.array(r.tests, dtype=np.int64), removed=np.array(r.removed, dtype=np.int64),
                near=near, near_p=near_p)


def make_large(procs):
    data, ar, alpha, md, _ = bnsynth.workload("large")
    r = oracle.pc_stable(data, ar, alpha, md)
    rec = _record(r, data.shape[0])
    out = os.path.join(HERE, "large_skeleton.npz")
    np.savez_compressed(out, n=data.shape[0], alpha=alpha, max_depth=md, **rec)
    return out, f"{len(rec['edges'])} edges, {len(rec['sep_pairs'])} non-empty separating sets, " \
                f"tests {list(rec['tests'])}, {len(rec['near'])} near-alpha tests"


_W = {}


def _depth0_init():
    _W["depth0"] = bnsynth.workload("depth0")


def _depth0_rows(args):
    lo, hi = args
    data, ar, alpha, _, _ = _W["depth0"]
    n = data.shape[0]
    keep, near = [], []
    for i in range(lo, hi):
        for j in range(i + 1, n):
            _, _, p = oracle.ci_test(data, ar, i, j)
            keep.append(not (p > alpha))
            if abs(p - alpha) <= 1e-6:
                near.append((i, j, p))
    return lo, keep, near


def make_depth0(procs):
    data, ar, alpha, md, _ = bnsynth.workload("depth0")
    n = data.shape[0]
    assert md == 0
    # blocks of rows with about equal pair counts
    bounds, acc, target = [0], 0, n * (n - 1) // 2 // (8 * procs)
    for i in range(n):
        acc += n - 1 - i
        if acc >= target:
            bounds.append(i + 1)
            acc = 0
    if bounds[-1] != n:
        bounds.append(n)
    with mp.get_context("spawn").Pool(procs, initializer=_depth0_init) as pool:
        parts = sorted(pool.map(_depth0_rows, list(zip(bounds[:-1], bounds[1:]))))
    keep = np.array([k for _, ks, _ in parts for k in ks], dtype=bool)
    near = [t for _, _, nr in parts for t in nr]
    assert keep.size == n * (n - 1) // 2
    out = os.path.join(HERE, "depth0_pairs.npz")
    np.savez_compressed(out, n=n, alpha=alpha, kept_bits=np.packbits(keep), n_pairs=keep.size,
                        near=np.array([(i, j) for i, j, _ in near], dtype=np.int32).reshape(-1, 2),
                        near_p=np.array([p for _, _, p in near], dtype=np.float64))
    return out, f"{int(keep.sum())} of {keep.size} pairs kept at depth 0, {len(near)} near-alpha tests"


def _batched_one(p):
    d, a, _ = bnsynth.batched_workload(1, first=p)[0]
    r = oracle.pc_stable(d, a, 0.05, -1)
    return p, d.shape[0], _record(r, d.shape[0])


BATCH_FIELDS = ("edges", "sep_pairs", "sep_lens", "sep_members", "tests", "removed", "near", "near_p")


def make_batched(procs, n_problems=256):
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        # largest problems first so that the pool ends evenly
        order = sorted(range(n_problems), key=lambda p: -np.prod(bnsynth.batched_size(p)))
        res = sorted(pool.imap_unordered(_batched_one, order))
    out = {"n_problems": n_problems, "alpha": 0.05, "max_depth": -1,
           "n": np.array([n for _, n, _ in res], dtype=np.int32)}
    small = {"edges": np.int16, "sep_pairs": np.int16, "sep_lens": np.int8, "sep_members": np.int16,
             "near": np.int16}   # n <= 300 variables per problem
    for f in BATCH_FIELDS:
        parts = [rec[f] for _, _, rec in res]
        out[f] = np.concatenate(parts) if parts else np.zeros(0)
        if f in small:
            assert out[f].size == 0 or int(np.abs(out[f]).max()) < np.iinfo(small[f]).max
            out[f] = out[f].astype(small[f])
        out[f + "_off"] = np.concatenate([[0], np.cumsum([len(x) for x in parts])]).astype(np.int64)
    path = os.path.join(HERE, "batched_skeletons.npz")
    np.savez_compressed(path, **out)
    n_near = int(out["near_off"][-1])
    return path, f"{n_problems} problems, {len(out['edges'])} edges kept, {len(out['sep_pairs'])} non-empty " \
                 f"separating sets, {int(out['tests'].sum())} tests, {n_near} near-alpha tests, " \
                 f"{time.time() - t0:.0f} s"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", nargs="?", default="large", choices=["large", "depth0", "batched"])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    t0 = time.time()
    path, what = {"large": make_large, "depth0": make_depth0, "batched": make_batched}[args.name](args.procs)
    print(f"{path}: {what} ({time.time() - t0:.0f} s, {args.procs} processes)")


if __name__ == "__main__":
    main()
