"""Pins of the oracle's CI-test variants: Pearson's X^2 (named with G^2 in
Section III-B) and degrees of freedom adjusted to the observed table.

X^2 is pinned to its closed form on 2x2 tables, to scipy's chi2_contingency
(without continuity correction, a library routine), to the sum over strata,
and to zero on an exactly independent table; the adjusted df to hand-counted
tables with empty rows, columns and strata; the composed test to the
survival function and to p = 1 when no degree of freedom is left; the
skeleton with the variants to the chain, fork and collider.
"""
import numpy as np
import pytest

import bnsynth
import oracle


def test_x2_closed_form_2x2():
    for a, b, c, d in [(10, 20, 30, 25), (1, 2, 3, 4), (50, 5, 7, 40), (0, 9, 4, 3)]:
        n = a + b + c + d
        want = n * (a * d - b * c) ** 2 / ((a + b) * (c + d) * (a + c) * (b + d))
        assert oracle.x2(np.array([a, b, c, d]), 2, 2) == pytest.approx(want, rel=1e-13)


def test_x2_matches_scipy_contingency():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(4)
    for _ in range(40):
        rx, ry = int(rng.integers(2, 6)), int(rng.integers(2, 6))
        t = rng.integers(1, 60, size=(rx, ry))
        want = scipy_stats.chi2_contingency(t, correction=False)[0]
        assert oracle.x2(t.ravel(), rx, ry) == pytest.approx(want, rel=1e-12)


def test_x2_sums_over_strata_and_vanishes_on_independence():
    s1 = np.array([10, 20, 30, 25]); s2 = np.array([3, 9, 14, 1])
    both = np.concatenate([s1, s2])
    assert oracle.x2(both, 2, 2) == pytest.approx(oracle.x2(s1, 2, 2) + oracle.x2(s2, 2, 2), rel=1e-13)
    indep = np.outer([1, 2, 3], [4, 5]) * 7          # N_xy = N_x N_y / N exactly
    assert oracle.x2(indep.ravel(), 3, 2) == 0.0
    # empty cells with E > 0 count: (0 - E)^2 / E = E
    assert oracle.x2(np.array([5, 0, 0, 5]), 2, 2) == pytest.approx(10.0, rel=1e-13)


def test_df_adjusted_counts_observed_rows_and_columns():
    full = np.arange(1, 13).reshape(3, 4)
    assert oracle.df_adjusted(full.ravel(), 3, 4) == 6                  # (3-1)(4-1)
    t = full.copy(); t[1, :] = 0                                         # an empty row
    assert oracle.df_adjusted(t.ravel(), 3, 4) == 3                     # (2-1)(4-1)
    t[:, 2] = 0                                                          # and an empty column
    assert oracle.df_adjusted(t.ravel(), 3, 4) == 2                     # (2-1)(3-1)
    strata = np.concatenate([full.ravel(), np.zeros(12, int), t.ravel()])
    assert oracle.df_adjusted(strata, 3, 4) == 6 + 0 + 2                 # an empty stratum adds nothing
    one_row = np.zeros((3, 4), int); one_row[0, :] = [1, 2, 3, 4]
    assert oracle.df_adjusted(one_row.ravel(), 3, 4) == 0


def test_ci_test_variants_compose():
    data, ar, *_ = bnsynth.workload("small")
    for S in [(), (2,), (3, 5)]:
        t = oracle.ci_table(data, ar, 0, 1, S)
        rx, ry = int(ar[0]), int(ar[1])
        for stat, f in (("g2", oracle.g2), ("x2", oracle.x2)):
            for mode in ("fixed", "adjusted"):
                st, df, p = oracle.ci_test(data, ar, 0, 1, S, stat=stat, df_mode=mode)
                assert st == pytest.approx(f(t, rx, ry), rel=1e-13)
                want_df = oracle.df(ar, 0, 1, S) if mode == "fixed" else oracle.df_adjusted(t, rx, ry)
                assert df == want_df
                assert p == pytest.approx(oracle.chisq_sf(int(df), st), rel=1e-13) if df > 0 else p == 1.0


def test_no_degree_of_freedom_cannot_reject():
    # X constant within the data: no observed variation, adjusted df = 0
    rng = np.random.default_rng(3)
    data = np.stack([np.zeros(500, np.uint8), rng.integers(0, 3, 500).astype(np.uint8)])
    ar = np.array([2, 3], np.uint8)
    for stat in ("g2", "x2"):
        st, df, p = oracle.ci_test(data, ar, 0, 1, stat=stat, df_mode="adjusted")
        assert df == 0 and p == 1.0 and st == 0.0


@pytest.mark.parametrize("stat,mode", [("x2", "fixed"), ("g2", "adjusted"), ("x2", "adjusted")])
def test_variant_skeletons_of_tiny_dags(stat, mode):
    for gen, edges, seps in [(bnsynth.chain, {(0, 1), (1, 2)}, {(0, 2): (1,)}),
                             (bnsynth.fork, {(0, 1), (1, 2)}, {(0, 2): (1,)}),
                             (bnsynth.collider, {(0, 2), (1, 2)}, {(0, 1): ()})]:
        data, ar = gen()
        r = oracle.pc_stable(data, ar, 0.05, -1, stat=stat, df_mode=mode)
        got = {(i, j) for i in range(3) for j in range(i + 1, 3) if r.adj[i, j]}
        assert got == edges and r.sepsets == seps
