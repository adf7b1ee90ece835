"""CPU oracle for PC-stable skeleton learning with the G^2 test.

TEST INFRASTRUCTURE ONLY: the plain, slow, sequential FP64 reference that the
GPU library is checked against.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the GPU library never
does, and the two share no code.

The arithmetic lives in ``fbn_oracle.c`` (plain C, compiled here with gcc on
first use); this module only marshals arguments.  Every function cites the
passage of the Fast-BNS paper it follows:

* ``ci_table``   -- contingency table, Section III-B / Section IV-A step (i);
* ``g2``         -- G^2 statistic and expected counts, Section III-B;
* ``x2``         -- Pearson's X^2 of the same table, Section III-B;
* ``df_adjusted``-- degrees of freedom of the observed table (skeleton variant);
* ``df``         -- degrees of freedom, Section III-B (conditional form);
* ``chisq_sf``   -- chi-square survival function, exact finite sums for integer df;
* ``ci_test``    -- one CI test and its decision rule, Section III-B;
* ``subsets``    -- conditioning sets in lexicographic order, Section IV-C;
* ``pc_stable``  -- Algorithm 1 with endpoint grouping (Section IV-C);
* ``orient_cpdag`` -- steps 2-3 of PC-stable (Section II-C): v-structures and
  Meek's rules, in ``cpdag.py`` (plain Python).

Parity is pinned for every function above by the CPU tests in
``tests/test_oracle_pins.py`` and ``tests/test_oracle_cpdag.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfbn_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fbn_oracle.c into a shared library (gcc, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i32, i64, f64, p = C.c_int32, C.c_int64, C.c_double, C.c_void_p
        lib.oracle_ci_table.restype = i64
        lib.oracle_ci_table.argtypes = [p, i64, i64, p, i32, i32, p, i32, p, i64]
        lib.oracle_g2.restype = f64
        lib.oracle_g2.argtypes = [p, i32, i32, i64]
        lib.oracle_df.restype = f64
        lib.oracle_df.argtypes = [p, i32, i32, p, i32]
        lib.oracle_chisq_sf.restype = f64
        lib.oracle_chisq_sf.argtypes = [i64, f64]
        lib.oracle_ci_test.restype = C.c_int
        lib.oracle_ci_test.argtypes = [p, i64, i64, p, i32, i32, p, i32, p, p, p]
        lib.oracle_ci_test_ex.restype = C.c_int
        lib.oracle_ci_test_ex.argtypes = [p, i64, i64, p, i32, i32, p, i32, i32, i32, p, p, p]
        lib.oracle_x2.restype = f64
        lib.oracle_x2.argtypes = [p, i32, i32, i64]
        lib.oracle_df_adjusted.restype = f64
        lib.oracle_df_adjusted.argtypes = [p, i32, i32, i64]
        lib.oracle_first_subset.restype = C.c_int
        lib.oracle_first_subset.argtypes = [i32, i32, p]
        lib.oracle_next_subset.restype = C.c_int
        lib.oracle_next_subset.argtypes = [i32, i32, p]
        lib.oracle_pc_stable.restype = p
        lib.oracle_pc_stable.argtypes = [p, i64, i32, i64, p, f64, i32, f64]
        lib.oracle_pc_stable_ex.restype = p
        lib.oracle_pc_stable_ex.argtypes = [p, i64, i32, i64, p, f64, i32, f64, i32, i32]
        lib.oracle_result_free.argtypes = [p]
        lib.oracle_result_adjacency.argtypes = [p, p]
        lib.oracle_result_sepset.restype = i32
        lib.oracle_result_sepset.argtypes = [p, i32, i32, p, i32]
        lib.oracle_result_depths.restype = i32
        lib.oracle_result_depths.argtypes = [p]
        lib.oracle_result_tests.restype = i64
        lib.oracle_result_tests.argtypes = [p, i32]
        lib.oracle_result_removed.restype = i64
        lib.oracle_result_removed.argtypes = [p, i32]
        lib.oracle_result_near_count.restype = i64
        lib.oracle_result_near_count.argtypes = [p]
        lib.oracle_result_near.argtypes = [p, p, p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _prep(data, arities):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    arities = np.ascontiguousarray(arities, dtype=np.uint8)
    assert data.ndim == 2 and arities.shape == (data.shape[0],)
    return data, arities


def ci_table(data, arities, x: int, y: int, S=()) -> np.ndarray:
    """Contingency table of I(X, Y | S) as int64, flat layout (z*r_x + x)*r_y + y,
    z mixed-radix over S with S[0] most significant (Section III-B)."""
    data, arities = _prep(data, arities)
    S = np.ascontiguousarray(S, dtype=np.int32)
    cells = int(arities[x]) * int(arities[y]) * int(np.prod([int(arities[s]) for s in S]) if len(S) else 1)
    out = np.zeros(cells, dtype=np.int64)
    got = _load().oracle_ci_table(_ptr(data), data.shape[1], data.shape[1], _ptr(arities), x, y,
                                  _ptr(S), len(S), _ptr(out), cells)
    assert got == cells
    return out


def g2(counts, rx: int, ry: int) -> float:
    """G^2 of a flat table with layout (z*rx + x)*ry + y (Section III-B)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64).ravel()
    assert counts.size % (rx * ry) == 0
    return _load().oracle_g2(_ptr(counts), rx, ry, counts.size // (rx * ry))


def x2(counts, rx: int, ry: int) -> float:
    """Pearson's X^2 of a flat table, layout as g2 (Section III-B names it next to G^2)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64).ravel()
    assert counts.size % (rx * ry) == 0
    return _load().oracle_x2(_ptr(counts), rx, ry, counts.size // (rx * ry))


def df_adjusted(counts, rx: int, ry: int) -> float:
    """Degrees of freedom of the observed table: sum over non-empty strata of
    (values of X seen - 1)(values of Y seen - 1)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64).ravel()
    assert counts.size % (rx * ry) == 0
    return _load().oracle_df_adjusted(_ptr(counts), rx, ry, counts.size // (rx * ry))


STATS = {"g2": 0, "x2": 1}
DF_MODES = {"fixed": 0, "adjusted": 1}


def df(arities, x: int, y: int, S=()) -> float:
    arities = np.ascontiguousarray(arities, dtype=np.uint8)
    S = np.ascontiguousarray(S, dtype=np.int32)
    return _load().oracle_df(_ptr(arities), x, y, _ptr(S), len(S))


def chisq_sf(k: int, x: float) -> float:
    """P(chi^2_k > x) for integer k >= 1."""
    return _load().oracle_chisq_sf(int(k), float(x))


def ci_test(data, arities, x: int, y: int, S=(), stat: str = "g2", df_mode: str = "fixed"):
    """(statistic, df, p) of I(X, Y | S) (Section III-B): G^2 or Pearson X^2,
    df from the declared arities or adjusted to the observed table (p = 1
    when no degree of freedom is left)."""
    data, arities = _prep(data, arities)
    S = np.ascontiguousarray(S, dtype=np.int32)
    out = np.zeros(3, dtype=np.float64)
    rc = _load().oracle_ci_test_ex(_ptr(data), data.shape[1], data.shape[1], _ptr(arities), x, y,
                                   _ptr(S), len(S), STATS[stat], DF_MODES[df_mode],
                                   _ptr(out[0:]), _ptr(out[1:]), _ptr(out[2:]))
    assert rc == 0
    return float(out[0]), float(out[1]), float(out[2])


def subsets(p: int, q: int):
    """All q-subsets of range(p) in the order the oracle enumerates them (Section IV-C)."""
    lib = _load()
    c = np.zeros(max(q, 1), dtype=np.int32)
    out = []
    if not lib.oracle_first_subset(p, q, _ptr(c)):
        return out
    while True:
        out.append(tuple(int(v) for v in c[:q]))
        if not lib.oracle_next_subset(p, q, _ptr(c)):
            return out


class PCResult:
    def __init__(self, adj, sepsets, tests, removed, near):
        self.adj = adj                  # uint8 [n][n]
        self.sepsets = sepsets          # {(i, j) with i<j removed: tuple(S)}
        self.tests = tests              # tests per depth
        self.removed = removed          # removals per depth
        self.near = near                # [(i, j, d, p)] tests with |p - alpha| <= near_tol

    @property
    def n_tests(self):
        return int(sum(self.tests))


def pc_stable(data, arities, alpha: float, max_depth: int = -1, near_tol: float = 1e-6, stat: str = "g2",
              df_mode: str = "fixed") -> PCResult:
    """PC-stable skeleton (Algorithm 1) with the grouping of Section IV-C;
    the CI test as in ci_test."""
    data, arities = _prep(data, arities)
    lib = _load()
    n, N = data.shape
    h = lib.oracle_pc_stable_ex(_ptr(data), N, n, N, _ptr(arities), float(alpha), int(max_depth),
                                float(near_tol), STATS[stat], DF_MODES[df_mode])
    if not h:
        raise MemoryError("oracle_pc_stable failed")
    try:
        adj = np.zeros((n, n), dtype=np.uint8)
        lib.oracle_result_adjacency(h, _ptr(adj))
        buf = np.zeros(n + 1, dtype=np.int32)
        sepsets = {}
        for i in range(n):
            for j in range(i + 1, n):
                k = lib.oracle_result_sepset(h, i, j, _ptr(buf), n + 1)
                if k >= 0:
                    sepsets[(i, j)] = tuple(int(v) for v in buf[:k])
        depths = lib.oracle_result_depths(h)
        tests = [int(lib.oracle_result_tests(h, d)) for d in range(depths)]
        removed = [int(lib.oracle_result_removed(h, d)) for d in range(depths)]
        nn = lib.oracle_result_near_count(h)
        ijd = np.zeros((max(nn, 1), 3), dtype=np.int32)
        pv = np.zeros(max(nn, 1), dtype=np.float64)
        if nn:
            lib.oracle_result_near(h, _ptr(ijd), _ptr(pv))
        near = [(int(ijd[k, 0]), int(ijd[k, 1]), int(ijd[k, 2]), float(pv[k])) for k in range(nn)]
    finally:
        lib.oracle_result_free(h)
    return PCResult(adj, sepsets, tests, removed, near)


from .cpdag import orient_cpdag  # noqa: E402
