"""Thin Python binding of libgpm (include/gpm.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does no
counting of its own: all enumeration runs in the CUDA kernels of libgpm.so.
If the library cannot be loaded the import-time ``load()`` raises; there is
no CPU fallback.

Arrays may be numpy (host) or torch tensors (host or CUDA); CUDA tensors are
passed to the library as device pointers (GPM_DEVICE_PTRS).  Streams may be a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None (the legacy
default stream).
"""
from __future__ import annotations

import ctypes
import gc
import os
import threading

import numpy as np

from . import build as _build

GPM_OK, GPM_EINVAL, GPM_ENOMEM, GPM_ECUDA, GPM_ETIMEOUT, GPM_EOVERFLOW, GPM_ENOTIMPL = range(7)
STATUS_NAMES = {0: "GPM_OK", 1: "GPM_EINVAL", 2: "GPM_ENOMEM", 3: "GPM_ECUDA", 4: "GPM_ETIMEOUT",
                5: "GPM_EOVERFLOW", 6: "GPM_ENOTIMPL"}
GPM_DEVICE_PTRS = 1
GPM_SKIP_VALIDATE = 2
GPM_APP_CLIQUE = 0
GPM_APP_MOTIF = 1
GPM_ORDER_ID = 0
GPM_ORDER_DEGREE_DESC = 1
GPM_ORDER_CUSTOM = 2
GPM_CLIQUE_MAX_K = 16
GPM_MOTIF_MAX_K = 8


class GpmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gpm_config(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("donate_min", ctypes.c_int32), ("order", ctypes.c_int32),
                ("max_idle_ms", ctypes.c_int32), ("donate", ctypes.c_int32),
                ("donate_after_us", ctypes.c_int32), ("clique_tail", ctypes.c_int32),
                ("clique_compact", ctypes.c_int32), ("motif_agg_min", ctypes.c_int32),
                ("clique_compact3", ctypes.c_int32), ("batch_split", ctypes.c_int32),
                ("clique_cpl", ctypes.c_int32)]


class gpm_monitor_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32), ("pad", ctypes.c_int32), ("spilled_units", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double), ("wall_ms", ctypes.c_double)]


class gpm_stats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_double), ("units_done", ctypes.c_uint64),
                ("donations", ctypes.c_uint64), ("idle_polls", ctypes.c_uint64),
                ("grid_blocks", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("word_ops", ctypes.c_uint64), ("kernel_launches", ctypes.c_int32),
                ("busy_warp_ns", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)

# int32 consumer(const int32* records, int64 count, int32 record_words, void* user)
GPM_LIST_CONSUMER = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_void_p)

# name -> (restype, argtypes); every symbol include/gpm.h declares
SIGNATURES = {
    "gpm_graph_create": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]),
    "gpm_graph_destroy": (None, [_vp]),
    "gpm_graph_info": (ctypes.c_int, [_vp, _i32p, _i64p, _i32p]),
    "gpm_clique_count": (ctypes.c_int, [_vp, ctypes.c_int, _u64p]),
    "gpm_clique_count_range": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u64p]),
    "gpm_motif_count": (ctypes.c_int, [_vp, ctypes.c_int, _u64p, ctypes.c_int64]),
    "gpm_motif_num_patterns": (ctypes.c_int, [ctypes.c_int, _i64p]),
    "gpm_motif_pattern": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _u64p]),
    "gpm_count_roots": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int64, _u64p,
                                       ctypes.c_int64, _u64p]),
    "gpm_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(gpm_config)]),
    "gpm_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(gpm_config)]),
    "gpm_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(gpm_stats)]),
    "gpm_last_error": (ctypes.c_char_p, []),
    "gpm_root_features": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_uint32]),
    "gpm_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp]),
    "gpm_mlp_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]),
    "gpm_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp, _vp]),
    "gpm_sched_from_scores": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _i32p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int32]),
    "gpm_count_scheduled": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u64p, ctypes.c_int64, _u64p]),
    "gpm_sched_balanced": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _i32p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int32]),
    "gpm_batch_create": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_uint32, _vp, ctypes.POINTER(_vp)]),
    "gpm_batch_destroy": (None, [_vp]),
    "gpm_batch_count": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u64p, _u64p]),
    "gpm_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(gpm_config), ctypes.POINTER(ctypes.c_double)]),
    "gpm_batch_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(gpm_config)]),
    "gpm_batch_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(gpm_stats)]),
    "gpm_motif_count_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int, _u64p, ctypes.c_int64, _vp]),
    "gpm_clique_count_dfs": (ctypes.c_int, [_vp, ctypes.c_int, _u64p]),
    "gpm_count_monitored": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _u64p, ctypes.c_int64,
                                           ctypes.POINTER(gpm_monitor_stats)]),
    "gpm_selftest_sum": (ctypes.c_int, [_u64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _u64p]),
    "gpm_measure_l2": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "gpm_list": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, GPM_LIST_CONSUMER,
                                ctypes.c_void_p, _u64p]),
}
GPM_MLP_PARAMS = 4801


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgpm.so (building it first if asked); raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libgpm is not built ({path}); run paper_2212_04551_gb300/build.py")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != GPM_OK:
        msg = load().gpm_last_error()
        raise GpmError(status, where, msg.decode() if msg else "")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _array_ptr(a, dtype):
    """(pointer, keepalive, is_device) for a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != (torch.int32 if dtype == np.int32 else torch.uint64):
                raise TypeError(f"expected {dtype}, got {a.dtype}")
            a = a.contiguous()
            return a.data_ptr(), a, a.is_cuda
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size == 0:
        arr = np.zeros(1, dtype=dtype)
    return arr.ctypes.data, arr, False


# listings in progress in this process (and whether the cyclic garbage
# collector was on before the first of them), and graphs whose destruction
# waits for them to end
_LISTING = [0, False]
_DEFERRED: list = []
_LISTING_LOCK = threading.Lock()


class Graph:
    """Owning handle of a gpm_graph (destroyed with the object)."""

    def __init__(self, handle: int, keep=()):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            if _LISTING[0]:
                # a listing kernel is running and waits for its consumer: a
                # destroy now (cudaFree waits for the device) would stall it,
                # so the handle is destroyed when the listing returns
                _DEFERRED.append(Graph(self.handle, self._keep))
            else:
                gpm_graph_destroy(self)
            self.handle = None

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


# ------------------------------------------------------------- entry points

def gpm_graph_create(indptr, indices, n: int | None = None, flags: int = 0, stream=None) -> Graph:
    lib = load()
    pi, ki, dev_i = _array_ptr(indptr, np.int32)
    px, kx, dev_x = _array_ptr(indices, np.int32)
    if dev_i != dev_x:
        raise ValueError("indptr and indices must both be host or both be device arrays")
    if dev_i:
        flags |= GPM_DEVICE_PTRS
    if n is None:
        n = int(indptr.shape[0]) - 1
    out = ctypes.c_void_p()
    st = lib.gpm_graph_create(pi, px, int(n), int(flags), _stream_handle(stream), ctypes.byref(out))
    _check(st, "gpm_graph_create")
    return Graph(out.value, keep=(ki, kx))


def gpm_graph_destroy(g: Graph) -> None:
    load().gpm_graph_destroy(ctypes.c_void_p(g.handle))


def gpm_graph_info(g: Graph) -> tuple[int, int, int]:
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    d = ctypes.c_int32()
    _check(load().gpm_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(d)), "gpm_graph_info")
    return n.value, m.value, d.value


def gpm_clique_count(g: Graph, k: int) -> int:
    out = ctypes.c_uint64()
    _check(load().gpm_clique_count(g, int(k), ctypes.byref(out)), "gpm_clique_count")
    return out.value


def gpm_clique_count_range(g: Graph, k_lo: int, k_hi: int) -> list[int]:
    out = (ctypes.c_uint64 * (k_hi - k_lo + 1))()
    _check(load().gpm_clique_count_range(g, int(k_lo), int(k_hi), out), "gpm_clique_count_range")
    return [int(x) for x in out]


def gpm_motif_num_patterns(k: int) -> int:
    out = ctypes.c_int64()
    _check(load().gpm_motif_num_patterns(int(k), ctypes.byref(out)), "gpm_motif_num_patterns")
    return out.value


def gpm_motif_pattern(k: int, pid: int) -> int:
    out = ctypes.c_uint64()
    _check(load().gpm_motif_pattern(int(k), int(pid), ctypes.byref(out)), "gpm_motif_pattern")
    return out.value


def gpm_motif_count(g: Graph, k: int) -> np.ndarray:
    npat = gpm_motif_num_patterns(k)
    out = np.zeros(npat, dtype=np.uint64)
    _check(load().gpm_motif_count(g, int(k), out.ctypes.data_as(_u64p), npat), "gpm_motif_count")
    return out


def gpm_count_roots(g: Graph, app: int, k: int, roots=None, per_root: bool = False):
    """Exact counts over a root subset: (counts, per_root or None)."""
    ncounts = 1 if app == GPM_APP_CLIQUE else gpm_motif_num_patterns(k)
    counts = np.zeros(ncounts, dtype=np.uint64)
    if roots is None:
        rp, nr = None, 0
        nrep = gpm_graph_info(g)[0]
    else:
        r = np.ascontiguousarray(roots, dtype=np.int32)
        rp, nr, nrep = r.ctypes.data_as(_i32p), int(r.shape[0]), int(r.shape[0])
    pr = np.zeros(max(nrep, 1), dtype=np.uint64) if per_root else None
    st = load().gpm_count_roots(g, int(app), int(k), rp, nr, counts.ctypes.data_as(_u64p), ncounts,
                                pr.ctypes.data_as(_u64p) if pr is not None else None)
    _check(st, "gpm_count_roots")
    return counts, (pr[:nrep] if pr is not None else None)


def gpm_clique_count_dfs(g: Graph, k: int) -> int:
    """k-cliques by the paper's DM_DFS baseline (one thread per root)."""
    out = ctypes.c_uint64()
    _check(load().gpm_clique_count_dfs(g, int(k), ctypes.byref(out)), "gpm_clique_count_dfs")
    return out.value


def gpm_list(g: Graph, app: int, k: int, consumer, pattern: int = -1, ring_records: int = 0) -> int:
    """List every k-clique (app CLIQUE) or connected induced k-subgraph (app
    MOTIF; ``pattern`` >= 0 lists that pattern's only) through the host ring.

    ``consumer(records)`` gets an int32 array of shape (count, k + 1) -- k
    vertex ids, then the pattern id (motifs) or -1 (cliques) -- valid during
    the call only (copy what you keep); returning True stops the listing.
    Returns the number of records delivered.  An exception raised by the
    consumer stops the listing and is raised again here."""
    errors = []

    def _cb(ptr, count, words, _user):
        try:
            arr = np.ctypeslib.as_array(ptr, shape=(int(count) * int(words),)).reshape(int(count), int(words))
            return 1 if consumer(arr) else 0
        except BaseException as e:  # noqa: BLE001 -- handed back to the caller below
            errors.append(e)
            return 1

    cb = GPM_LIST_CONSUMER(_cb)
    out = ctypes.c_uint64()
    # The consumer runs while the kernel runs and waits for it, so nothing on
    # this thread may wait for the device meanwhile: no cyclic garbage
    # collection (finalizers of unreachable graphs would free device memory,
    # and cudaFree waits for the device), and graphs released during the
    # call are destroyed after it.
    with _LISTING_LOCK:
        if _LISTING[0] == 0:
            _LISTING[1] = gc.isenabled()
            gc.disable()
        _LISTING[0] += 1
    try:
        st = load().gpm_list(g, int(app), int(k), int(pattern), int(ring_records), cb, None, ctypes.byref(out))
    finally:
        with _LISTING_LOCK:
            _LISTING[0] -= 1
            last = _LISTING[0] == 0
            if last and _LISTING[1]:
                gc.enable()
        if last:
            while _DEFERRED:
                _DEFERRED.pop().close()
    if errors:
        raise errors[0]
    _check(st, "gpm_list")
    return out.value


def gpm_count_monitored(g: Graph, app: int, k: int, threshold: float):
    """Counts under the paper's host-monitored stop / redistribute / restart
    balancing: (counts, stats dict)."""
    ncounts = 1 if app == GPM_APP_CLIQUE else gpm_motif_num_patterns(k)
    counts = np.zeros(ncounts, dtype=np.uint64)
    st = gpm_monitor_stats()
    _check(load().gpm_count_monitored(g, int(app), int(k), float(threshold), counts.ctypes.data_as(_u64p), ncounts,
                                      ctypes.byref(st)), "gpm_count_monitored")
    return counts, {f: getattr(st, f) for f, _ in gpm_monitor_stats._fields_ if f != "pad"}


def gpm_get_config(g: Graph) -> gpm_config:
    c = gpm_config()
    _check(load().gpm_get_config(g, ctypes.byref(c)), "gpm_get_config")
    return c


def gpm_set_config(g: Graph, cfg: gpm_config | None = None, **kw) -> None:
    c = cfg if cfg is not None else gpm_get_config(g)
    for key, val in kw.items():
        setattr(c, key, int(val))
    _check(load().gpm_set_config(g, ctypes.byref(c)), "gpm_set_config")


def _stats_dict(s: gpm_stats) -> dict:
    d = {f: getattr(s, f) for f, _ in gpm_stats._fields_}
    slots = d["grid_blocks"] * d["warps_per_block"] * d["kernel_ms"] * 1e6
    # fraction of the grid's warp-time spent without a work unit
    d["idle_warp_frac"] = max(0.0, 1.0 - d["busy_warp_ns"] / slots) if slots > 0 else None
    return d


def gpm_get_stats(g: Graph) -> dict:
    s = gpm_stats()
    _check(load().gpm_get_stats(g, ctypes.byref(s)), "gpm_get_stats")
    return _stats_dict(s)


def gpm_last_error() -> str:
    m = load().gpm_last_error()
    return m.decode() if m else ""


def graph_from_csr(csr, stream=None, flags: int = 0) -> Graph:
    """Create a device graph from a ``graphs.CSR`` (host arrays)."""
    return gpm_graph_create(csr.indptr, csr.indices, csr.n, flags=flags, stream=stream)


# ------------------------------------------------------- learned scheduler

def _dev_ptr(t, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def gpm_root_features(g: Graph, k: int, out=None):
    """Per-vertex FP32 features [n][8] for size k; into ``out`` (CUDA tensor) or a new host array."""
    n = gpm_graph_info(g)[0]
    if out is None:
        arr = np.zeros((max(n, 1), 8), dtype=np.float32)
        _check(load().gpm_root_features(g, int(k), arr.ctypes.data, 0), "gpm_root_features")
        return arr[:n]
    _check(load().gpm_root_features(g, int(k), _dev_ptr(out, "out"), GPM_DEVICE_PTRS), "gpm_root_features")
    return out


def gpm_mlp_forward(w_bf16, x, y, stream=None) -> None:
    n = int(x.shape[0])
    _check(load().gpm_mlp_forward(_dev_ptr(w_bf16, "w"), _dev_ptr(x, "x"), n, _dev_ptr(y, "y"),
                                  _stream_handle(stream)), "gpm_mlp_forward")


def gpm_mlp_grad(w_bf16, x, t, grad, loss, stream=None) -> None:
    n = int(x.shape[0])
    _check(load().gpm_mlp_grad(_dev_ptr(w_bf16, "w"), _dev_ptr(x, "x"), _dev_ptr(t, "t"), n,
                               _dev_ptr(grad, "grad"), _dev_ptr(loss, "loss"), _stream_handle(stream)),
           "gpm_mlp_grad")


def gpm_mlp_adam(master, m, v, grad, step: int, lr: float, w_bf16, stream=None) -> None:
    _check(load().gpm_mlp_adam(_dev_ptr(master, "master"), _dev_ptr(m, "m"), _dev_ptr(v, "v"),
                               _dev_ptr(grad, "grad"), int(step), float(lr), _dev_ptr(w_bf16, "w"),
                               _stream_handle(stream)), "gpm_mlp_adam")


def gpm_sched_from_scores(g: Graph, app: int, scores=None, roots=None, split_roots: int = 0,
                          split_chunks: int = 0) -> None:
    sp = _dev_ptr(scores, "scores") if scores is not None else None
    if roots is None:
        rp, nr = None, 0
    else:
        r = np.ascontiguousarray(roots, dtype=np.int32)
        rp, nr = r.ctypes.data_as(_i32p), int(r.shape[0])
    _check(load().gpm_sched_from_scores(g, int(app), sp, rp, nr, int(split_roots), int(split_chunks)),
           "gpm_sched_from_scores")


def gpm_sched_balanced(g: Graph, app: int, scores, roots=None, target_units: int = 16384,
                       max_chunks: int = 64) -> None:
    sp = _dev_ptr(scores, "scores")
    if roots is None:
        rp, nr = None, 0
    else:
        r = np.ascontiguousarray(roots, dtype=np.int32)
        rp, nr = r.ctypes.data_as(_i32p), int(r.shape[0])
    _check(load().gpm_sched_balanced(g, int(app), sp, rp, nr, int(target_units), int(max_chunks)),
           "gpm_sched_balanced")


def gpm_count_scheduled(g: Graph, app: int, k: int, n_roots: int | None = None, per_root: bool = False):
    ncounts = 1 if app == GPM_APP_CLIQUE else gpm_motif_num_patterns(k)
    counts = np.zeros(ncounts, dtype=np.uint64)
    pr = None
    if per_root:
        if n_roots is None:
            raise ValueError("per_root needs n_roots (the length of the scheduled root list)")
        pr = np.zeros(max(n_roots, 1), dtype=np.uint64)
    _check(load().gpm_count_scheduled(g, int(app), int(k), counts.ctypes.data_as(_u64p), ncounts,
                                      pr.ctypes.data_as(_u64p) if pr is not None else None),
           "gpm_count_scheduled")
    return counts, (pr[:n_roots] if pr is not None else None)


# ------------------------------------------------------- batched launch

class Batch:
    """Owning handle of a gpm_batch."""

    def __init__(self, handle: int, n_graphs: int, keep=()):
        self.handle = handle
        self.n_graphs = n_graphs
        self._keep = keep

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().gpm_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


def gpm_batch_create(graph_off, indptr, indices, flags: int = 0, stream=None) -> Batch:
    lib = load()
    pg, kg, dg_ = _array_ptr(graph_off, np.int32)
    pi, ki, di = _array_ptr(indptr, np.int32)
    px, kx, dx = _array_ptr(indices, np.int32)
    if not (dg_ == di == dx):
        raise ValueError("all arrays must be host or all device")
    if di:
        flags |= GPM_DEVICE_PTRS
    n_graphs = int(graph_off.shape[0]) - 1
    out = ctypes.c_void_p()
    _check(lib.gpm_batch_create(pg, pi, px, n_graphs, int(flags), _stream_handle(stream), ctypes.byref(out)),
           "gpm_batch_create")
    return Batch(out.value, n_graphs, keep=(kg, ki, kx))


def gpm_batch_destroy(b: Batch) -> None:
    b.close()


def gpm_batch_count(b: Batch, clique_k: int, motif_k: int):
    """(clique counts [G] or None, motif counts [G, P] or None)."""
    G = b.n_graphs
    cc = np.zeros(max(G, 1), dtype=np.uint64) if clique_k else None
    npat = gpm_motif_num_patterns(motif_k) if motif_k else 0
    mc = np.zeros((max(G, 1), max(npat, 1)), dtype=np.uint64) if motif_k else None
    _check(load().gpm_batch_count(b, int(clique_k), int(motif_k),
                                  cc.ctypes.data_as(_u64p) if cc is not None else None,
                                  mc.ctypes.data_as(_u64p) if mc is not None else None), "gpm_batch_count")
    return (cc[:G] if cc is not None else None), (mc[:G, :npat] if mc is not None else None)


def gpm_batch_autotune(b: Batch, clique_k: int, motif_k: int, reps: int = 3):
    c = gpm_config()
    ms = ctypes.c_double()
    _check(load().gpm_batch_autotune(b, int(clique_k), int(motif_k), int(reps), ctypes.byref(c), ctypes.byref(ms)),
           "gpm_batch_autotune")
    return {f: getattr(c, f) for f, _ in gpm_config._fields_}, ms.value


def gpm_batch_set_config(b: Batch, **kw) -> None:
    c = gpm_config()
    c.warps_per_block = 0
    c.donate_min = 4
    c.order = GPM_ORDER_DEGREE_DESC
    c.max_idle_ms = 120000
    c.donate = 1
    c.donate_after_us = 50
    c.motif_agg_min = 16
    c.clique_compact3 = 1
    c.batch_split = 1
    c.clique_cpl = 85
    for key, val in kw.items():
        setattr(c, key, int(val))
    _check(load().gpm_batch_set_config(b, ctypes.byref(c)), "gpm_batch_set_config")


def gpm_batch_get_stats(b: Batch) -> dict:
    s = gpm_stats()
    _check(load().gpm_batch_get_stats(b, ctypes.byref(s)), "gpm_batch_get_stats")
    return _stats_dict(s)


def batch_from_graphs(graph_list, stream=None) -> Batch:
    """Pack a list of ``graphs.CSR`` (local ids) into one batch (global ids)."""
    goff = np.zeros(len(graph_list) + 1, dtype=np.int64)
    goff[1:] = np.cumsum([g.n for g in graph_list])
    ip_parts = [np.zeros(1, dtype=np.int64)]
    ix_parts = []
    eoff = 0
    for g, base in zip(graph_list, goff[:-1]):
        ip_parts.append(g.indptr[1:].astype(np.int64) + eoff)
        ix_parts.append(g.indices.astype(np.int64) + base)
        eoff += g.indices.shape[0]
    indptr = np.concatenate(ip_parts).astype(np.int32)
    indices = (np.concatenate(ix_parts) if ix_parts else np.zeros(0, dtype=np.int64)).astype(np.int32)
    return gpm_batch_create(goff.astype(np.int32), indptr, indices, stream=stream)


def gpm_motif_count_noalloc(indptr, indices, n: int, k: int, stream=None) -> np.ndarray:
    """Allocation-free motif counting on a graph already on the device
    (CUDA int32 tensors); see include/gpm.h for the limits."""
    npat = gpm_motif_num_patterns(k)
    out = np.zeros(npat, dtype=np.uint64)
    _check(load().gpm_motif_count_noalloc(_dev_ptr(indptr, "indptr"), _dev_ptr(indices, "indices") if
                                          indices.numel() else None, int(n), int(k), out.ctypes.data_as(_u64p),
                                          npat, _stream_handle(stream)), "gpm_motif_count_noalloc")
    return out


def gpm_selftest_sum(values, blocks: int = 1, threads: int = 32) -> int:
    """Exact device sum of uint64 values through the kernels' carry-checked
    reduction path (GpmError with GPM_EOVERFLOW when it exceeds 2^64-1)."""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    out = ctypes.c_uint64()
    _check(load().gpm_selftest_sum(v.ctypes.data_as(_u64p), int(v.shape[0]), int(blocks), int(threads),
                                   ctypes.byref(out)), "gpm_selftest_sum")
    return out.value


def gpm_measure_l2(nbytes: int = 64 << 20, mode: int = 0, reps: int = 20) -> float:
    """L2 read bandwidth in GB/s (mode 0 coalesced, mode 1 random 32-byte sectors)."""
    out = ctypes.c_double()
    _check(load().gpm_measure_l2(int(nbytes), int(mode), int(reps), ctypes.byref(out)), "gpm_measure_l2")
    return out.value
