"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Counts must be bit-exact; G^2 within 1e-6 relative and p within 1e-9 absolute
of the FP64 oracle; skeletons and separating sets identical except for
differences traceable to tests whose oracle p-value lies within 1e-6 of alpha.
"""
import numpy as np
import pytest

import bnsynth
import oracle
from _compare import compare

pytestmark = pytest.mark.gpu

G2_REL, P_ABS = 1e-6, 1e-9


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


def _rand(seed, arities, N):
    rng = np.random.default_rng(seed)
    ar = np.asarray(arities, dtype=np.uint8)
    return np.stack([rng.integers(0, r, N) for r in ar]).astype(np.uint8), ar


def _tests(rng, n, dmax, count):
    out = []
    for _ in range(count):
        d = int(rng.integers(0, dmax + 1))
        v = rng.permutation(n)[: d + 2]
        out.append((int(v[0]), int(v[1]), [int(t) for t in v[2:]]))
    return out


@pytest.mark.parametrize("N", [1, 15, 16, 17, 255, 1000, 4099, 65537])
def test_tables_bit_exact_ragged(F, N):
    data, ar = _rand(N, [2, 3, 4, 5, 2, 3, 4, 5, 3], N)
    h = F.fbn_create(data, ar)
    rng = np.random.default_rng(100 + N)
    for x, y, S in _tests(rng, len(ar), 4, 25):
        got = F.fbn_ci_table(h, x, y, S)
        ref = oracle.ci_table(data, ar, x, y, S)
        assert np.array_equal(got[: ref.size], ref), (x, y, S)
        assert int(got[: ref.size].sum()) == N


@pytest.mark.parametrize("cells_target", ["lane", "warp", "cta", "global"])
def test_tables_every_count_strategy(F, cells_target):
    # table sizes that land in each shared/global counting strategy
    shapes = {"lane": [3, 4, 5], "warp": [16, 16, 8], "cta": [16, 16, 32], "global": [16, 16, 16, 16]}
    arities = shapes[cells_target] + [2]
    data, ar = _rand(7, arities, 30011)
    h = F.fbn_create(data, ar)
    k = len(shapes[cells_target])
    x, y, S = 0, 1, list(range(2, k))
    got = F.fbn_ci_table(h, x, y, S)
    ref = oracle.ci_table(data, ar, x, y, S)
    assert np.array_equal(got[: ref.size], ref)
    g2, df, p = F.fbn_ci_test(h, x, y, S)
    rg2, rdf, rp = oracle.ci_test(data, ar, x, y, S)
    assert df == rdf
    assert g2 == pytest.approx(rg2, rel=G2_REL)
    assert abs(p - rp) <= P_ABS


def test_ci_test_matches_oracle_on_workloads(F):
    for name, count in [("small", 120), ("mid", 60)]:
        data, ar, *_ = bnsynth.workload(name)
        h = F.fbn_create(data, ar)
        rng = np.random.default_rng(11)
        for x, y, S in _tests(rng, len(ar), 4, count):
            g2, df, p = F.fbn_ci_test(h, x, y, S)
            rg2, rdf, rp = oracle.ci_test(data, ar, x, y, S)
            assert df == rdf
            assert g2 == pytest.approx(rg2, rel=G2_REL, abs=1e-12), (x, y, S)
            assert abs(p - rp) <= P_ABS, (x, y, S, p, rp)


def test_degenerate_tables(F):
    # constant column (declared arity 3, only value 0 occurs): G^2 = 0, p = 1,
    # df still uses the declared arity; a single sample
    data, ar = _rand(3, [3, 2, 4], 5000)
    data[0] = 0
    h = F.fbn_create(data, ar)
    g2, df, p = F.fbn_ci_test(h, 0, 1, [2])
    assert g2 == 0.0 and p == 1.0 and df == 2 * 1 * 4
    one, ar1 = _rand(4, [2, 2, 2], 1)
    h1 = F.fbn_create(one, ar1)
    assert F.fbn_ci_test(h1, 0, 1, [2])[0] == 0.0
    assert int(F.fbn_ci_table(h1, 0, 1, [2]).sum()) == 1


def test_z_order_defines_layout(F):
    data, ar = _rand(9, [2, 3, 4, 5], 999)
    h = F.fbn_create(data, ar)
    for S in ([2, 3], [3, 2]):
        assert np.array_equal(F.fbn_ci_table(h, 0, 1, S)[:120], oracle.ci_table(data, ar, 0, 1, S))
    a, b = F.fbn_ci_test(h, 0, 1, [2, 3]), F.fbn_ci_test(h, 0, 1, [3, 2])
    assert a[0] == pytest.approx(b[0], rel=1e-12) and a[1] == b[1]


def _skeleton(F, data, ar, alpha, md, **opt):
    h = F.fbn_create(data, ar, **opt)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    return h, adj, F.fbn_export_sepsets(h), F.fbn_get_stats(h)


@pytest.mark.parametrize("opt", [dict(form="pool"), dict(form="pool", group_size=1),
                                 dict(form="pool", group_size=4),
                                 dict(form="pool", group_size=9), dict(form="plain"),
                                 dict(form="pool", group_threads=32),
                                 dict(form="pool", group_threads=64),
                                 dict(form="pool", group_threads=128, group_size=2),
                                 dict(form="pool", depth1="tensor"),
                                 dict(form="pool", group_threads=256, group_size=3)])
@pytest.mark.parametrize("name", ["small", "mid"])
def test_skeleton_parity(F, name, opt):
    data, ar, alpha, md, _ = bnsynth.workload(name)
    ref = oracle.pc_stable(data, ar, alpha, md)
    h, adj, sep, st = _skeleton(F, data, ar, alpha, md, **opt)
    hard, excused, cascade = compare(adj, sep, ref)
    assert not hard, hard[:5]
    assert np.array_equal(adj, adj.T) and not adj.diagonal().any()
    if not ref.near:
        # oracle-equivalent test count per depth equals the sequential count
        assert st["tests_oracle"] == ref.tests
        assert st["removed"] == ref.removed
        assert all(t >= o for t, o in zip(st["tests"], st["tests_oracle"]))
    for (i, j), S in sep.items():
        assert F.fbn_get_sepset(h, i, j) == S


def test_tiny_dags(F):
    for gen, edges, sepsets in [(bnsynth.chain, {(0, 1), (1, 2)}, {(0, 2): (1,)}),
                                (bnsynth.fork, {(0, 1), (1, 2)}, {(0, 2): (1,)}),
                                (bnsynth.collider, {(0, 2), (1, 2)}, {(0, 1): ()})]:
        data, ar = gen()
        h, adj, sep, _ = _skeleton(F, data, ar, 0.05, -1)
        got = {(i, j) for i in range(3) for j in range(i + 1, 3) if adj[i, j]}
        assert got == edges and sep == sepsets


def test_max_depth_and_alpha(F):
    data, ar, alpha, _, _ = bnsynth.workload("small")
    for md, a in [(0, 0.05), (1, 0.05), (2, 0.01), (-1, 0.2)]:
        ref = oracle.pc_stable(data, ar, a, md)
        _, adj, sep, st = _skeleton(F, data, ar, a, md)
        hard, _, _ = compare(adj, sep, ref)
        assert not hard
        assert st["depths"] == len(ref.tests)


def test_batch_matches_individual(F):
    probs = bnsynth.batched_workload(6, first=0, n_range=(20, 45), samples_range=(1000, 8000))
    hs = [F.fbn_create(d, a) for d, a, _ in probs]
    adjs = F.fbn_learn_skeleton_batch(hs, 0.05, -1)
    for (d, a, _), h, adj in zip(probs, hs, adjs):
        ref = oracle.pc_stable(d, a, 0.05, -1)
        hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
        assert not hard


def test_device_resident_input_and_output(F):
    import torch
    data, ar, alpha, md, _ = bnsynth.workload("small")
    h = F.fbn_create(torch.from_numpy(data).cuda(), ar)
    out = torch.zeros((len(ar), len(ar)), dtype=torch.uint8, device="cuda")
    F.fbn_learn_skeleton(h, alpha, md, adj_out=out)
    ref = oracle.pc_stable(data, ar, alpha, md)
    assert np.array_equal(out.cpu().numpy(), ref.adj)


def test_errors(F):
    data, ar = _rand(1, [2, 3, 4], 100)
    bad = data.copy()
    bad[1, 57] = 3
    with pytest.raises(F.FbnError) as e:
        F.fbn_create(bad, ar)
    assert e.value.code == -2 and "sample 57" in str(e.value)
    h = F.fbn_create(data, ar)
    for args in [(0, 0, []), (0, 1, [1]), (0, 1, [2, 2]), (0, 5, []), (-1, 1, [])]:
        with pytest.raises(F.FbnError) as e:
            F.fbn_ci_test(h, *args)
        assert e.value.code == -1
    with pytest.raises(F.FbnError):
        F.fbn_learn_skeleton(h, 1.5, -1)
    big, arb = _rand(2, [255, 255, 255, 2], 50)
    hb = F.fbn_create(big, arb)
    with pytest.raises(F.FbnError) as e:
        F.fbn_ci_test(hb, 0, 1, [2, 3])
    assert e.value.code == -5


def test_update_data(F):
    a_data, a_ar, alpha, md, _ = bnsynth.workload("small")
    rng = np.random.default_rng(77)
    b_data = np.stack([rng.integers(0, r, a_data.shape[1]) for r in a_ar]).astype(np.uint8)
    h = F.fbn_create(a_data, a_ar)
    F.fbn_learn_skeleton(h, alpha, md)
    F.fbn_update_data(h, b_data)
    adj = F.fbn_learn_skeleton(h, alpha, md)
    ref = oracle.pc_stable(b_data, a_ar, alpha, md)
    hard, _, _ = compare(adj, F.fbn_export_sepsets(h), ref)
    assert not hard
    assert F.fbn_ci_test(h, 0, 1, [2])[0] == pytest.approx(oracle.ci_test(b_data, a_ar, 0, 1, [2])[0], rel=1e-6)
    bad = b_data.copy()
    bad[3, 11] = a_ar[3]
    with pytest.raises(F.FbnError) as e:
        F.fbn_update_data(h, bad)
    assert e.value.code == -2
