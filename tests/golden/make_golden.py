"""Write the oracle's skeleton of the large workload as a golden file.

Runs only the CPU oracle on the seeded large workload (1000 variables, 1200
edges, 100,000 samples, alpha 0.01, depth <= 4) and stores what the GPU parity
test compares at full size: the remaining edges, every non-empty separating
set (removed pairs not listed have the empty set), the tests and removals per
depth, and the tests whose p-value lies within 1e-6 of alpha.

    python tests/golden/make_golden.py        # takes a few minutes
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bnsynth  # noqa: E402
import oracle   # noqa: E402


def main(name="large"):
    data, ar, alpha, md, _ = bnsynth.workload(name)
    t0 = time.time()
    r = oracle.pc_stable(data, ar, alpha, md)
    n = data.shape[0]
    edges = np.array([(i, j) for i in range(n) for j in range(i + 1, n) if r.adj[i, j]], dtype=np.int32)
    nonempty = sorted((k, v) for k, v in r.sepsets.items() if len(v) > 0)
    pairs = np.array([k for k, _ in nonempty], dtype=np.int32).reshape(-1, 2)
    lens = np.array([len(v) for _, v in nonempty], dtype=np.int32)
    members = np.array([m for _, v in nonempty for m in v], dtype=np.int32)
    near = np.array([(i, j, d) for (i, j, d, _) in r.near], dtype=np.int32).reshape(-1, 3)
    near_p = np.array([p for (_, _, _, p) in r.near], dtype=np.float64)
    out = os.path.join(HERE, f"{name}_skeleton.npz")
    np.savez_compressed(out, n=n, alpha=alpha, max_depth=md, edges=edges, sep_pairs=pairs, sep_lens=lens,
                        sep_members=members, tests=np.array(r.tests, dtype=np.int64),
                        removed=np.array(r.removed, dtype=np.int64), near=near, near_p=near_p)
    print(f"{out}: {len(edges)} edges, {len(pairs)} non-empty separating sets, tests {r.tests}, "
          f"{len(r.near)} near-alpha tests, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(*sys.argv[1:])
