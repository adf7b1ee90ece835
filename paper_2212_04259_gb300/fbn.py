"""ctypes binding of libfbn (include/fbn.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers, checks status codes and raises ``FbnError``.
There is no CPU fallback: importing works without a GPU, but every call needs
the built library and a CUDA device, and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfbn.so")

FBN_OK, FBN_EINVAL, FBN_EDATA, FBN_ENOMEM, FBN_ECUDA, FBN_ETOOBIG, FBN_ETIMEOUT, FBN_ENUMERIC = \
    0, -1, -2, -3, -4, -5, -6, -7
FORMS = {"pool": 0, "plain": 1}
DEPTH0 = {"auto": 0, "hist": 1, "gram": 2}
DEPTH1 = {"auto": 0, "pool": 1, "tensor": 2}
STATISTIC = {"g2": 0, "x2": 1}
DF_MODE = {"fixed": 0, "adjusted": 1}
LOOP = {"device": 0, "host": 1}
COUNT = {"auto": 0, "hist": 1, "bits": 2}
TUNE = {"off": 0, "auto": 1}
MAX_DEPTHS = 64

# Every symbol include/fbn.h declares.
EXPORTS = ("fbn_create", "fbn_set_stream", "fbn_ci_test", "fbn_ci_table", "fbn_learn_skeleton",
           "fbn_learn_skeleton_batch", "fbn_get_sepset", "fbn_export_sepsets", "fbn_orient_cpdag", "fbn_get_stats",
           "fbn_last_error", "fbn_destroy", "fbn_ci_test_noalloc", "fbn_pairwise_counts",
           "fbn_update_data", "fbn_measure_unit_rates", "fbn_autotune", "fbn_learn_skeleton_sharded",
           "fbn_update_data_batch")

# Callback types of fbn_learn_skeleton_sharded (include/fbn.h).
OWN_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_uint8), C.POINTER(C.c_uint8))
EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64),
                          C.c_int64, C.POINTER(C.c_int64))


class FbnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fbn error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("form", C.c_int32), ("group_size", C.c_int32), ("depth0", C.c_int32),
                ("device", C.c_int32), ("group_threads", C.c_int32), ("wait_limit", C.c_int32),
                ("depth1", C.c_int32), ("statistic", C.c_int32), ("df_mode", C.c_int32),
                ("loop", C.c_int32), ("count", C.c_int32), ("tune", C.c_int32), ("reserved", C.c_int32 * 4)]


class Tuning(C.Structure):
    _fields_ = [("depths", C.c_int32), ("depth0", C.c_int32), ("group_threads", C.c_int32 * MAX_DEPTHS),
                ("count", C.c_int32 * MAX_DEPTHS), ("ms_fixed", C.c_double), ("ms_tuned", C.c_double),
                ("candidates", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("depths", C.c_int32), ("reserved", C.c_int32), ("launches", C.c_int64),
                ("edges", C.c_int64 * MAX_DEPTHS), ("tests", C.c_int64 * MAX_DEPTHS),
                ("tests_oracle", C.c_int64 * MAX_DEPTHS), ("removed", C.c_int64 * MAX_DEPTHS),
                ("ms", C.c_double * MAX_DEPTHS), ("test_ms", C.c_double * MAX_DEPTHS),
                ("gram_ms", C.c_double), ("gram_rows", C.c_int64), ("gram_samples", C.c_int64),
                ("test_samples", C.c_int64 * MAX_DEPTHS), ("popc_work", C.c_int64 * MAX_DEPTHS),
                ("smem_updates", C.c_int64 * MAX_DEPTHS)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libfbn.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfbn.so is not built ({LIB_PATH}); run "
                               "`python -m paper_2212_04259_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        p, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.fbn_create.restype = C.c_int
        L.fbn_create.argtypes = [p, i32, i64, p, p, C.POINTER(p)]
        L.fbn_set_stream.restype = C.c_int
        L.fbn_set_stream.argtypes = [p, p]
        L.fbn_ci_test.restype = C.c_int
        L.fbn_ci_test.argtypes = [p, i32, i32, p, i32, p, p, p]
        L.fbn_ci_table.restype = C.c_int
        L.fbn_ci_table.argtypes = [p, i32, i32, p, i32, p, i64]
        L.fbn_learn_skeleton.restype = C.c_int
        L.fbn_learn_skeleton.argtypes = [p, f64, i32, p]
        L.fbn_learn_skeleton_batch.restype = C.c_int
        L.fbn_learn_skeleton_batch.argtypes = [p, i32, f64, i32, p]
        L.fbn_get_sepset.restype = i32
        L.fbn_get_sepset.argtypes = [p, i32, i32, p, i32]
        L.fbn_export_sepsets.restype = C.c_int
        L.fbn_export_sepsets.argtypes = [p, p, p, p, p, p]
        L.fbn_get_stats.restype = C.c_int
        L.fbn_get_stats.argtypes = [p, p]
        L.fbn_orient_cpdag.restype = C.c_int
        L.fbn_orient_cpdag.argtypes = [p, p]
        L.fbn_last_error.restype = C.c_char_p
        L.fbn_last_error.argtypes = [p]
        L.fbn_destroy.restype = None
        L.fbn_destroy.argtypes = [p]
        L.fbn_update_data.restype = C.c_int
        L.fbn_update_data.argtypes = [p, p]
        L.fbn_update_data_batch.restype = C.c_int
        L.fbn_update_data_batch.argtypes = [p, i32, p]
        L.fbn_pairwise_counts.restype = C.c_int
        L.fbn_pairwise_counts.argtypes = [p, p, i64]
        L.fbn_learn_skeleton_sharded.restype = C.c_int
        L.fbn_learn_skeleton_sharded.argtypes = [p, f64, i32, OWN_FN, EXCHANGE_FN, p, p]
        L.fbn_autotune.restype = C.c_int
        L.fbn_autotune.argtypes = [p, i32, f64, i32, p]
        L.fbn_measure_unit_rates.restype = C.c_int
        L.fbn_measure_unit_rates.argtypes = [i32, p, i32]
        L.fbn_ci_test_noalloc.restype = C.c_int
        L.fbn_ci_test_noalloc.argtypes = [p, i64, i32, i64, p, i32, i32, p, i32, p, p, p]
        _lib = L
        return L


def _check(rc, h=None):
    if rc != FBN_OK:
        msg = lib().fbn_last_error(h.ptr if h is not None else None)
        raise FbnError(rc, msg.decode() if msg else "")


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(C.c_void_p)
    return C.c_void_p(x.data_ptr())


def _need_out(t, name, np_dtype, numel):
    """Check a caller-owned output buffer before its address goes to a C entry
    point that writes numel elements there without knowing the buffer's size:
    a numpy array or torch tensor (host or device) of np_dtype, contiguous,
    writable, with at least numel elements.  Raises ValueError otherwise."""
    if isinstance(t, np.ndarray):
        ok = t.dtype == np_dtype and t.flags.c_contiguous and t.flags.writeable and t.size >= numel
    else:
        try:
            import torch
        except ImportError:
            torch = None
        ok = (torch is not None and isinstance(t, torch.Tensor) and t.is_contiguous() and t.numel() >= numel
              and t.dtype == {np.uint8: torch.uint8, np.int32: torch.int32}[np_dtype])
    if not ok:
        raise ValueError(f"{name} must be a contiguous, writable {np.dtype(np_dtype).name} array or tensor "
                         f"of at least {numel} elements")


class Handle:
    """An fbn_handle*; destroyed on garbage collection or by fbn_destroy."""

    def __init__(self, ptr, n, n_samples, arities):
        self.ptr = ptr
        self.n = n
        self.n_samples = n_samples
        self.arities = arities
        self._keep = None

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().fbn_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _as_u8_2d(data):
    if isinstance(data, np.ndarray):
        data = np.ascontiguousarray(data, dtype=np.uint8)
        return data, data.shape
    import torch  # torch tensors: host or device memory
    if data.dtype != torch.uint8 or data.dim() != 2:
        raise ValueError("data must be a 2-D uint8 tensor [n_vars][n_samples]")
    data = data.contiguous()
    return data, tuple(data.shape)


def fbn_create(data, arities, form="pool", group_size=0, depth0="auto", device=-1,
               group_threads=0, wait_limit=0, depth1="auto", statistic="g2", df="fixed",
               loop="device", count="auto", tune="off") -> Handle:
    """Upload variable-major uint8 data [n_vars][n_samples] (numpy, or torch host/device)."""
    data, (n, N) = _as_u8_2d(data)
    ar = np.ascontiguousarray(arities, dtype=np.uint8)
    if ar.shape != (n,):
        raise ValueError("arities must have one entry per variable")
    o = Options(form=FORMS[form], group_size=group_size, depth0=DEPTH0[depth0], device=device,
                group_threads=group_threads, wait_limit=wait_limit, depth1=DEPTH1[depth1],
                statistic=STATISTIC[statistic], df_mode=DF_MODE[df], loop=LOOP[loop], count=COUNT[count],
                tune=TUNE[tune])
    out = C.c_void_p()
    rc = lib().fbn_create(_ptr(data), n, N, _ptr(ar), C.byref(o), C.byref(out))
    _check(rc)
    return Handle(out, n, N, ar.copy())


def fbn_update_data(h: Handle, data) -> None:
    """Replace the samples (same shape) from numpy or a torch host/device tensor."""
    data, shape = _as_u8_2d(data)
    if tuple(shape) != (h.n, h.n_samples):
        raise ValueError("data must keep the handle's shape")
    _check(lib().fbn_update_data(h.ptr, _ptr(data)), h)


def fbn_update_data_batch(handles, datas) -> None:
    """fbn_update_data on every handle at once (one synchronisation)."""
    k = len(handles)
    if len(datas) != k:
        raise ValueError("one data set per handle")
    keep = []
    for hh, d in zip(handles, datas):
        d, shape = _as_u8_2d(d)
        if tuple(shape) != (hh.n, hh.n_samples):
            raise ValueError("data must keep the handle's shape")
        keep.append(d)
    arr = (C.c_void_p * k)(*[hh.ptr.value if isinstance(hh.ptr, C.c_void_p) else hh.ptr for hh in handles])
    dp = (C.c_void_p * k)(*[_ptr(d).value for d in keep])
    _check(lib().fbn_update_data_batch(C.cast(arr, C.c_void_p), k, C.cast(dp, C.c_void_p)), handles[0])


def fbn_set_stream(h: Handle, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None."""
    if stream is None:
        raw = None
    elif isinstance(stream, int):
        raw = stream
    else:
        raw = stream.cuda_stream
    _check(lib().fbn_set_stream(h.ptr, C.c_void_p(raw) if raw else None), h)


def _zarr(z):
    return np.ascontiguousarray(list(z), dtype=np.int32)


def fbn_ci_test(h: Handle, x: int, y: int, z=()):
    """(G^2, df, p) of I(X, Y | Z)."""
    za = _zarr(z)
    g2, df, p = C.c_double(), C.c_double(), C.c_double()
    _check(lib().fbn_ci_test(h.ptr, x, y, _ptr(za) if len(za) else None, len(za), C.byref(g2),
                             C.byref(df), C.byref(p)), h)
    return g2.value, df.value, p.value


def fbn_ci_table(h: Handle, x: int, y: int, z=(), cells=None) -> np.ndarray:
    """Exact int32 contingency table, layout (zi * r_x + xv) * r_y + yv."""
    za = _zarr(z)
    if cells is None:
        cells = int(h.arities[x]) * int(h.arities[y])
        for v in za:
            cells *= int(h.arities[v]) if 0 <= v < h.n else 1
        cells = max(1, min(cells, 1 << 25))
    out = np.zeros(cells, dtype=np.int32)
    _check(lib().fbn_ci_table(h.ptr, x, y, _ptr(za) if len(za) else None, len(za), _ptr(out), cells), h)
    return out


def fbn_pairwise_counts(h: Handle, out=None) -> np.ndarray:
    """All depth-0 pair tables as the symmetric int32 [M][M] one-hot Gram
    (M = sum of arities); out may be a preallocated host or device buffer."""
    M = int(sum(int(a) for a in h.arities))
    if out is None:
        out = np.zeros((M, M), dtype=np.int32)
    _need_out(out, "out", np.int32, M * M)
    _check(lib().fbn_pairwise_counts(h.ptr, _ptr(out), M * M), h)
    return out


def fbn_learn_skeleton(h: Handle, alpha: float, max_depth: int = -1, adj_out=None):
    """Skeleton adjacency. adj_out: None (a numpy array is returned), or a
    preallocated uint8 [n][n] numpy array / torch tensor (host or device)."""
    out = np.zeros((h.n, h.n), dtype=np.uint8) if adj_out is None else adj_out
    _need_out(out, "adj_out", np.uint8, h.n * h.n)
    _check(lib().fbn_learn_skeleton(h.ptr, float(alpha), int(max_depth), _ptr(out)), h)
    return out


def fbn_learn_skeleton_batch(handles, alpha: float, max_depth: int = -1, adj_out=None):
    k = len(handles)
    arr = (C.c_void_p * k)(*[hh.ptr.value if isinstance(hh.ptr, C.c_void_p) else hh.ptr for hh in handles])
    outs = [np.zeros((hh.n, hh.n), dtype=np.uint8) for hh in handles] if adj_out is None else adj_out
    if len(outs) != k:
        raise ValueError("adj_out must hold one buffer per handle")
    for p, (hh, o) in enumerate(zip(handles, outs)):
        _need_out(o, f"adj_out[{p}]", np.uint8, hh.n * hh.n)
    optr = (C.c_void_p * k)(*[_ptr(o).value for o in outs])
    rc = lib().fbn_learn_skeleton_batch(C.cast(arr, C.c_void_p), k, float(alpha), int(max_depth),
                                        C.cast(optr, C.c_void_p))
    _check(rc, handles[0])
    return outs


def fbn_learn_skeleton_sharded(h: Handle, alpha: float, max_depth: int, own, exchange, adj_out=None):
    """The skeleton learnt together with other processes (include/fbn.h).

    own(depth, adj) -> uint8/bool [n][n]: the edges (entries i < j) this
    process tests at that depth, given the shared graph adj (uint8 [n][n]).
    exchange(depth, local) -> int64 [M][3]: every process's (i, j, rank)
    removal records of the depth, given this process's (int64 [m][3])."""
    n = h.n
    errors = []

    def _own(_ctx, depth, n_, adj_p, owned_p):
        try:
            adj = np.ctypeslib.as_array(adj_p, shape=(n_, n_)).copy()
            mask = np.ascontiguousarray(own(int(depth), adj), dtype=np.uint8)
            if mask.shape != (n_, n_):
                raise ValueError("own must return an [n][n] mask")
            np.ctypeslib.as_array(owned_p, shape=(n_, n_))[:] = mask
            return 0
        except Exception as e:   # reported after the call
            errors.append(e)
            return 1

    def _exchange(_ctx, depth, local_p, n_local, all_p, cap, n_all_p):
        try:
            local = np.ctypeslib.as_array(local_p, shape=(int(n_local), 3)).copy() if n_local else \
                np.zeros((0, 3), dtype=np.int64)
            every = np.ascontiguousarray(exchange(int(depth), local), dtype=np.int64).reshape(-1, 3)
            if len(every) > cap:
                raise ValueError("more removal records than edges")
            if len(every):
                np.ctypeslib.as_array(all_p, shape=(int(cap), 3))[: len(every)] = every
            n_all_p[0] = len(every)
            return 0
        except Exception as e:
            errors.append(e)
            return 1

    own_c, exch_c = OWN_FN(_own), EXCHANGE_FN(_exchange)
    out = np.zeros((n, n), dtype=np.uint8) if adj_out is None else adj_out
    _need_out(out, "adj_out", np.uint8, n * n)
    rc = lib().fbn_learn_skeleton_sharded(h.ptr, float(alpha), int(max_depth), own_c, exch_c, None, _ptr(out))
    if errors:
        raise errors[0]
    _check(rc, h)
    return out


def fbn_autotune(handles, alpha: float, max_depth: int = -1) -> dict:
    """Measure the candidate configurations on these handles and keep per depth
    the fastest (see include/fbn.h); returns the choices."""
    k = len(handles)
    arr = (C.c_void_p * k)(*[hh.ptr.value if isinstance(hh.ptr, C.c_void_p) else hh.ptr for hh in handles])
    t = Tuning()
    _check(lib().fbn_autotune(C.cast(arr, C.c_void_p), k, float(alpha), int(max_depth), C.byref(t)), handles[0])
    d = t.depths
    return {"depths": d, "depth0": {1: "hist", 2: "gram"}.get(t.depth0, "auto"),
            "group_threads": list(t.group_threads[:d]),
            "count": [{1: "hist", 2: "bits"}.get(c, "auto") for c in t.count[:d]],
            "ms_fixed": t.ms_fixed, "ms_tuned": t.ms_tuned, "candidates": t.candidates}


def fbn_get_sepset(h: Handle, i: int, j: int):
    """Separating set of (i, j) as a tuple, or None while adjacent."""
    buf = np.zeros(64, dtype=np.int32)
    k = lib().fbn_get_sepset(h.ptr, i, j, _ptr(buf), len(buf))
    if k == -1:
        return None
    if k < -1:
        _check(k, h)
    if k > len(buf):   # the call reports the full size; read again with room for it
        buf = np.zeros(k, dtype=np.int32)
        k = lib().fbn_get_sepset(h.ptr, i, j, _ptr(buf), len(buf))
        if k < 0:
            _check(k, h)
    return tuple(int(v) for v in buf[:k])


def fbn_export_sepsets(h: Handle, as_dict: bool = True):
    """{(i, j): tuple(S)} for every removed pair i < j; with as_dict=False the
    CSR arrays (pairs int32 [R][2], offsets int64 [R+1], members int32)."""
    nr, nm = C.c_int64(), C.c_int64()
    L = lib()
    _check(L.fbn_export_sepsets(h.ptr, C.byref(nr), C.byref(nm), None, None, None), h)
    pairs = np.zeros((max(nr.value, 1), 2), dtype=np.int32)
    offs = np.zeros(nr.value + 1, dtype=np.int64)
    mem = np.zeros(max(nm.value, 1), dtype=np.int32)
    _check(L.fbn_export_sepsets(h.ptr, C.byref(nr), C.byref(nm), _ptr(pairs), _ptr(offs), _ptr(mem)), h)
    if not as_dict:
        return pairs[: nr.value], offs, mem[: nm.value]
    return {(int(pairs[k, 0]), int(pairs[k, 1])): tuple(int(v) for v in mem[offs[k]:offs[k + 1]])
            for k in range(nr.value)}


def fbn_orient_cpdag(h: Handle) -> np.ndarray:
    """CPDAG of the last skeleton (v-structures + Meek rules): uint8 [n][n],
    M[a][b] = 1, M[b][a] = 0 for a -> b; both 1 for an undirected edge."""
    out = np.zeros((h.n, h.n), dtype=np.uint8)
    _check(lib().fbn_orient_cpdag(h.ptr, _ptr(out)), h)
    return out


def fbn_get_stats(h: Handle) -> dict:
    s = Stats()
    _check(lib().fbn_get_stats(h.ptr, C.byref(s)), h)
    d = s.depths
    return {"depths": d, "launches": int(s.launches), "edges": list(s.edges[:d]),
            "tests": list(s.tests[:d]), "tests_oracle": list(s.tests_oracle[:d]),
            "removed": list(s.removed[:d]), "ms": list(s.ms[:d]), "test_ms": list(s.test_ms[:d]),
            "gram_ms": float(s.gram_ms), "gram_rows": int(s.gram_rows), "gram_samples": int(s.gram_samples),
            "test_samples": list(s.test_samples[:d]), "popc_work": list(s.popc_work[:d]),
            "smem_updates": list(s.smem_updates[:d])}


def fbn_last_error(h: Handle | None = None) -> str:
    m = lib().fbn_last_error(h.ptr if h is not None else None)
    return m.decode() if m else ""


def fbn_measure_unit_rates(device: int = -1) -> dict:
    """Measured shared-memory reduction and POPC throughput of the device."""
    out = np.zeros(4, dtype=np.float64)
    _check(lib().fbn_measure_unit_rates(int(device), _ptr(out), 4))
    return {"smem_red_per_s": float(out[0]), "popc_per_s": float(out[1]), "sms": int(out[2]),
            "sm_clock_hz": float(out[3])}


def fbn_destroy(h: Handle) -> None:
    if h.ptr:
        lib().fbn_destroy(h.ptr)
        h.ptr = None


def fbn_ci_test_noalloc(data_dev, ld: int, n_samples: int, arities, x: int, y: int, z, out_dev,
                        table_dev=None, stream=None) -> None:
    """Enqueue one CI test on caller-owned device buffers, allocating nothing.

    data_dev: device uint8 tensor holding [n_vars][ld] rows; out_dev: device
    float64 tensor of 3 (G^2, df, p), written in stream order; table_dev:
    optional device int32 tensor for the counts.  stream: torch.cuda.Stream,
    raw handle or None (the legacy default stream)."""
    import torch
    ar = np.ascontiguousarray(arities, dtype=np.uint8)
    za = _zarr(z)
    n_vars = len(ar)
    dev = torch.cuda.current_device()

    def need(t, name, dtype, numel):
        # the C entry point reads and writes these buffers without knowing their sizes
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.device.index != dev:
            raise ValueError(f"{name} must be a tensor on the current CUDA device (cuda:{dev})")
        if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of at least {numel} elements")

    need(data_dev, "data_dev", torch.uint8, n_vars * int(ld))
    need(out_dev, "out_dev", torch.float64, 3)
    if table_dev is not None:
        cells = int(ar[x]) * int(ar[y]) * int(np.prod([int(ar[v]) for v in za], dtype=np.int64)) \
            if all(0 <= v < n_vars for v in list(za) + [x, y]) else 0
        need(table_dev, "table_dev", torch.int32, cells)
    raw = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    rc = lib().fbn_ci_test_noalloc(_ptr(data_dev), int(ld), len(ar), int(n_samples), _ptr(ar), x, y,
                                   _ptr(za) if len(za) else None, len(za), _ptr(out_dev),
                                   _ptr(table_dev), C.c_void_p(raw) if raw else None)
    _check(rc)
