"""fbn_ci_test_noalloc: the CI test for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator (a framework's caching allocator) or to a budget fixed at start-up,
or their loop must not stall in an allocation.  The entry point runs the test
on buffers the caller owns, with one fixed scratch array inside the library.

Checked here against the CPU oracle and against fbn_ci_test, within the
tolerances of the other GPU tests (table bit-exact, G^2 within 1e-6
relative, p within 1e-9 absolute), on two calls in a row (the scratch array
keeps the previous call's contents); with several calls queued on one stream
without synchronising; with device memory unchanged across calls; and with
a value out of range, which must give NaN outputs and leave the context
usable.  The big table below does not fit in shared memory, so it goes
through the scratch array.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

G2_REL, P_ABS = 1e-6, 1e-9


@pytest.fixture(scope="module")
def F():
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as f
    return f


def _data(N=30011, seed=2026):
    rng = np.random.default_rng(seed)
    ar = np.array([16, 16, 16, 16, 3, 2, 5], dtype=np.uint8)
    data = np.stack([rng.integers(0, r, N) for r in ar]).astype(np.uint8)
    return data, ar


def _device_rows(data):
    import torch
    n, N = data.shape
    ld = (N + 255) // 256 * 256
    dev = torch.zeros((n, ld), dtype=torch.uint8, device="cuda")
    dev[:, :N] = torch.from_numpy(data).cuda()
    return dev, ld


CASES = [(0, 1, [2, 3]),      # 65,536 cells: through the scratch array
         (4, 5, [6]),         # small table: shared memory only
         (0, 4, [5, 1])]


def _cells(ar, x, y, S):
    return int(ar[x]) * int(ar[y]) * int(np.prod([int(ar[s]) for s in S]))


def test_noalloc_matches_oracle_and_ci_test(F):
    import torch
    data, ar = _data()
    N = data.shape[1]
    h = F.fbn_create(data, ar)
    dev, ld = _device_rows(data)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for _ in range(2):            # two calls in a row for every case
        for x, y, S in CASES:
            table = torch.full((_cells(ar, x, y, S),), -7, dtype=torch.int32, device="cuda")
            F.fbn_ci_test_noalloc(dev, ld, N, ar, x, y, S, out, table, torch.cuda.current_stream())
            torch.cuda.synchronize()
            g2, df, p = out.tolist()
            og2, odf, op = oracle.ci_test(data, ar, x, y, S)
            assert df == odf
            assert g2 == pytest.approx(og2, rel=G2_REL, abs=1e-12)
            assert abs(p - op) <= P_ABS
            assert np.array_equal(table.cpu().numpy(), oracle.ci_table(data, ar, x, y, S))
            rg2, rdf, rp = F.fbn_ci_test(h, x, y, S)
            assert df == rdf and g2 == pytest.approx(rg2, rel=G2_REL, abs=1e-12) and abs(p - rp) <= P_ABS


def test_noalloc_queued_on_one_stream_allocates_nothing(F):
    import torch
    data, ar = _data(N=20000, seed=7)
    N = data.shape[1]
    dev, ld = _device_rows(data)
    st = torch.cuda.Stream()
    outs = [torch.zeros(3, dtype=torch.float64, device="cuda") for _ in range(3 * len(CASES))]
    tables = [torch.zeros(_cells(ar, *CASES[k % len(CASES)]), dtype=torch.int32, device="cuda")
              for k in range(len(outs))]
    torch.cuda.synchronize()
    # a warm call does the per-device set-up; afterwards no call may change
    # the device's free memory or torch's allocation
    F.fbn_ci_test_noalloc(dev, ld, N, ar, *CASES[0], outs[0], tables[0], st)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(len(outs)):    # queued back to back, no synchronisation between them
        x, y, S = CASES[k % len(CASES)]
        F.fbn_ci_test_noalloc(dev, ld, N, ar, x, y, S, outs[k], tables[k], st)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    for k in range(len(outs)):
        x, y, S = CASES[k % len(CASES)]
        g2, df, p = outs[k].tolist()
        og2, odf, op = oracle.ci_test(data, ar, x, y, S)
        assert df == odf and g2 == pytest.approx(og2, rel=G2_REL, abs=1e-12) and abs(p - op) <= P_ABS
        assert np.array_equal(tables[k].cpu().numpy(), oracle.ci_table(data, ar, x, y, S))


def test_noalloc_value_out_of_range_gives_nan(F):
    import torch
    data, ar = _data(N=5003, seed=3)
    N = data.shape[1]
    dev, ld = _device_rows(data)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for row, col in ((2, 4099), (1, N - 1)):      # inside a 16-sample vector, and in the ragged tail
        bad = dev.clone()
        bad[row, col] = int(ar[row])               # one value equal to its arity
        table = torch.full((_cells(ar, 0, 1, [2, 3]),), -7, dtype=torch.int32, device="cuda")
        F.fbn_ci_test_noalloc(bad, ld, N, ar, 0, 1, [2, 3], out, table)
        torch.cuda.synchronize()
        assert all(np.isnan(v) for v in out.tolist())
        assert bool((table == -7).all())           # nothing written
    # the context stays usable and the next call is exact again
    F.fbn_ci_test_noalloc(dev, ld, N, ar, 0, 1, [2, 3], out)
    torch.cuda.synchronize()
    g2, df, p = out.tolist()
    og2, odf, op = oracle.ci_test(data, ar, 0, 1, [2, 3])
    assert df == odf and g2 == pytest.approx(og2, rel=G2_REL, abs=1e-12) and abs(p - op) <= P_ABS


def test_noalloc_rejects_tables_over_its_limit(F):
    import torch
    ar = np.array([64, 64, 64, 2], dtype=np.uint8)   # 64^3 = 262,144 cells fit, x2 does not
    dev = torch.zeros((4, 256), dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FbnError) as e:
        F.fbn_ci_test_noalloc(dev, 256, 100, ar, 0, 1, [2, 3], out)
    assert e.value.code == -5
    F.fbn_ci_test_noalloc(dev, 256, 100, ar, 0, 1, [2], out)
    torch.cuda.synchronize()
    assert out[0].item() == 0.0 and out[2].item() == 1.0   # all-zero data: one occupied cell
