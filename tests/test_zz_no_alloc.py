"""fbn_ci_test_noalloc against fbn_ci_test.

The no-allocation entry point serves callers that cannot allocate device
memory (their memory belongs to another allocator or a fixed budget, or
allocation would stall a latency-critical loop).  It must give the same
table, G^2, df and p as the ordinary entry point, within the tolerances the
other GPU tests use, on two calls in a row (its fixed scratch array keeps the
previous call's contents and must be cleared by each call).  The big table
below does not fit in shared memory, so it runs through that scratch array.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

G2_REL, P_ABS = 1e-6, 1e-9


def test_noalloc_matches_ci_test():
    import torch
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as F

    rng = np.random.default_rng(2026)
    ar = np.array([16, 16, 16, 16, 3, 2, 5], dtype=np.uint8)
    N = 30011
    data = np.stack([rng.integers(0, r, N) for r in ar]).astype(np.uint8)
    h = F.fbn_create(data, ar)
    ld = (N + 255) // 256 * 256
    dev = torch.zeros((len(ar), ld), dtype=torch.uint8, device="cuda")
    dev[:, :N] = torch.from_numpy(data).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    cases = [(0, 1, [2, 3]),      # 65,536 cells: through the scratch array
             (4, 5, [6]),         # small table: shared memory only
             (0, 4, [5, 1])]
    for _ in range(2):            # two calls in a row for every case
        for x, y, S in cases:
            cells = int(ar[x]) * int(ar[y]) * int(np.prod([int(ar[s]) for s in S]))
            table = torch.full((cells,), -7, dtype=torch.int32, device="cuda")
            F.fbn_ci_test_noalloc(dev, ld, N, ar, x, y, S, out, table, torch.cuda.current_stream())
            torch.cuda.synchronize()
            g2, df, p = out.tolist()
            rg2, rdf, rp = F.fbn_ci_test(h, x, y, S)
            assert df == rdf
            assert g2 == pytest.approx(rg2, rel=G2_REL, abs=1e-12)
            assert abs(p - rp) <= P_ABS
            assert np.array_equal(table.cpu().numpy(), F.fbn_ci_table(h, x, y, S))


def test_noalloc_rejects_tables_over_its_limit():
    import torch
    from paper_2212_04259_gb300 import build
    build.build()
    import paper_2212_04259_gb300 as F

    ar = np.array([64, 64, 64, 2], dtype=np.uint8)   # 64^3 = 262,144 cells fit, x2 does not
    dev = torch.zeros((4, 256), dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FbnError) as e:
        F.fbn_ci_test_noalloc(dev, 256, 100, ar, 0, 1, [2, 3], out)
    assert e.value.code == -5
    F.fbn_ci_test_noalloc(dev, 256, 100, ar, 0, 1, [2], out)
    torch.cuda.synchronize()
    assert out[0].item() == 0.0 and out[2].item() == 1.0   # all-zero data: one occupied cell
