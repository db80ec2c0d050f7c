"""Thin ctypes binding of libpilot (include/pilot.h): argument marshalling only.

Every step of a search runs in the library's CUDA kernels.  Arrays may be
numpy arrays (host memory) or torch tensors (host or CUDA); torch is used only
to hold device memory and streams.  If libpilot.so is missing this module
raises on import: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PILOT_LIBRARY selects another build of the same library (e.g. the checked one)
LIB_PATH = os.environ.get("PILOT_LIBRARY") or os.path.join(_HERE, "libpilot.so")

PILOT_OK, PILOT_EINVAL, PILOT_ENOMEM, PILOT_ECUDA, PILOT_EIO, PILOT_ETIMEOUT, PILOT_EBUSY, PILOT_EFORMAT = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EIO", "ETIMEOUT", "EBUSY", "EFORMAT"]
METRIC_L2, METRIC_IP = 0, 1
FULL_VECS_DEVICE, FULL_VECS_HOST = 0, 1
LOAD_FULL_VECS_HOST = 1
REDUCED_CODES = {"f32": 0, "bf16": 1, "fp8": 2}
PILOT_MAX_EF = 512

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libpilot.so not built ({LIB_PATH}); run paper_2503_21206_b300/build.py")
_lib = ctypes.CDLL(LIB_PATH)


class PilotError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"PILOT_{name}: {message}")


class pilot_index_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("dp", ctypes.c_int64), ("R", ctypes.c_int64),
                ("R_sub", ctypes.c_int64), ("n_entry", ctypes.c_int64), ("metric", ctypes.c_int32),
                ("reduced_dtype", ctypes.c_int32), ("graph", ctypes.c_void_p), ("subgraph_mask", ctypes.c_void_p),
                ("subgraph", ctypes.c_void_p), ("svd_basis", ctypes.c_void_p), ("reduced_vecs", ctypes.c_void_p),
                ("reduced_scales", ctypes.c_void_p), ("full_vecs", ctypes.c_void_p), ("entry_ids", ctypes.c_void_p),
                ("full_vecs_location", ctypes.c_int32), ("n_clusters", ctypes.c_int64),
                ("entry_cluster", ctypes.c_void_p), ("cluster_centroids", ctypes.c_void_p)]


class pilot_search_options(ctypes.Structure):
    _fields_ = [("stage1", ctypes.c_int32), ("stage2_expansions", ctypes.c_int32), ("stage3", ctypes.c_int32),
                ("use_fes", ctypes.c_int32), ("warps_per_block", ctypes.c_int32), ("stage_rows", ctypes.c_int32),
                ("counters", ctypes.c_void_p), ("kernel_ms", ctypes.c_void_p), ("status_words", ctypes.c_void_p),
                ("fes_seeds", ctypes.c_int32), ("seed_ids", ctypes.c_void_p), ("seed_count", ctypes.c_int32),
                ("visited_entries", ctypes.c_int32)]


_P = ctypes.c_void_p
_lib.pilot_last_error.restype = ctypes.c_char_p
_lib.pilot_abi_version.restype = ctypes.c_int
_lib.pilot_index_load.argtypes = [ctypes.POINTER(pilot_index_desc), ctypes.POINTER(_P)]
_lib.pilot_index_load_files.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(_P)]
_lib.pilot_index_free.argtypes = [_P]
_lib.pilot_index_free.restype = None
_lib.pilot_index_info.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int64)] * 5
_lib.pilot_search_options_default.argtypes = [ctypes.POINTER(pilot_search_options)]
_lib.pilot_search_options_default.restype = None
_lib.pilot_search.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P, _P]
_lib.pilot_search_noalloc.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P, _P]
PILOT_NOALLOC_SCRATCH_BYTES = 16 << 20
_lib.pilot_search_ex.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                 ctypes.POINTER(pilot_search_options)]


def pilot_last_error() -> str:
    return _lib.pilot_last_error().decode()


def pilot_abi_version() -> int:
    return _lib.pilot_abi_version()


def _check(status: int):
    if status != PILOT_OK:
        raise PilotError(status, pilot_last_error())


def _addr(a):
    """Raw address of a numpy array or torch tensor (must be C-contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libpilot must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors passed to libpilot must be contiguous")
    return a.data_ptr()


def _dtype_name(a) -> str:
    """'float32', 'int32', ... for a numpy array or a torch tensor."""
    return a.dtype.name if isinstance(a, np.ndarray) else str(a.dtype).split(".")[-1]


def _numel(a) -> int:
    return int(a.size) if isinstance(a, np.ndarray) else int(a.numel())


def _device_of(a):
    """None for host memory, else the CUDA device index."""
    if isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False):
        return None
    return a.device.index


def _check_search_buffers(index, queries, k: int, out_ids, out_dists, counters=None):
    """Reject, before any pointer reaches the library, buffers whose type or
    size would let a kernel read or write past them."""
    d = index.dim
    if _dtype_name(queries) != "float32" or len(queries.shape) != 2 or int(queries.shape[1]) != d:
        raise ValueError(f"queries must be float32 of shape (nq, {d}); got {_dtype_name(queries)} "
                         f"{tuple(queries.shape)}")
    nq = int(queries.shape[0])
    for name, a, dt, need in (("out_ids", out_ids, "int32", nq * k), ("out_dists", out_dists, "float32", nq * k),
                              ("counters", counters, "int32", nq * 8)):
        if a is None:
            continue
        if _dtype_name(a) != dt:
            raise ValueError(f"{name} must be {dt}, got {_dtype_name(a)}")
        if _numel(a) < need:
            raise ValueError(f"{name} holds {_numel(a)} elements; nq x {need // max(nq, 1)} = {need} are written")


def pilot_search_options_default() -> pilot_search_options:
    o = pilot_search_options()
    _lib.pilot_search_options_default(ctypes.byref(o))
    return o


class PilotIndex:
    """Owns a pilot_index handle (device memory held by the library)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        self._dim = None

    @property
    def dim(self) -> int:
        """Dimension d of the index's vectors."""
        if self._dim is None:
            self._dim = int(self.info()["d"])
        return self._dim

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        vals = [ctypes.c_int64() for _ in range(5)]
        _check(_lib.pilot_index_info(self._h, *[ctypes.byref(v) for v in vals]))
        return dict(zip(["n", "d", "dp", "n_sub", "device_bytes"], [v.value for v in vals]))

    def free(self):
        if self._h:
            _lib.pilot_index_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def pilot_index_load(graph, subgraph_mask, subgraph, svd_basis, reduced_vecs, full_vecs, entry_ids, *,
                     metric: int = METRIC_L2, reduced_dtype: str = "f32", reduced_scales=None,
                     full_vecs_host: bool = False, entry_cluster=None, cluster_centroids=None) -> PilotIndex:
    """Copy an index (host numpy arrays, layouts as in pilot.h) to the current device.
    ``full_vecs_host`` keeps the full vectors in pinned host memory instead;
    ``entry_cluster`` / ``cluster_centroids`` enable the clustered FES."""
    if _device_of(full_vecs) is not None:   # a CUDA tensor: the library copies from device memory
        if _dtype_name(full_vecs) != "float32" or len(full_vecs.shape) != 2 or not full_vecs.is_contiguous():
            raise ValueError("full_vecs on the device must be a contiguous float32 (n, d) tensor")
        fv = full_vecs
    else:
        fv = np.ascontiguousarray(full_vecs, np.float32)
    arrs = dict(graph=np.ascontiguousarray(graph, np.int32), subgraph_mask=np.ascontiguousarray(subgraph_mask, np.uint8),
                subgraph=np.ascontiguousarray(subgraph, np.int32),
                svd_basis=np.ascontiguousarray(svd_basis, np.float64),
                reduced_vecs=np.ascontiguousarray(reduced_vecs),
                full_vecs=fv,
                entry_ids=np.ascontiguousarray(entry_ids, np.int32))
    sc = None if reduced_scales is None else np.ascontiguousarray(reduced_scales, np.float32)
    ec = None if entry_cluster is None else np.ascontiguousarray(entry_cluster, np.int32)
    cc = None if cluster_centroids is None else np.ascontiguousarray(cluster_centroids, np.float32)
    n, d = arrs["full_vecs"].shape
    desc = pilot_index_desc(n=n, d=d, dp=arrs["svd_basis"].shape[1], R=arrs["graph"].shape[1],
                            R_sub=arrs["subgraph"].shape[1], n_entry=arrs["entry_ids"].shape[0], metric=metric,
                            reduced_dtype=REDUCED_CODES[reduced_dtype], graph=_addr(arrs["graph"]),
                            subgraph_mask=_addr(arrs["subgraph_mask"]), subgraph=_addr(arrs["subgraph"]),
                            svd_basis=_addr(arrs["svd_basis"]), reduced_vecs=_addr(arrs["reduced_vecs"]),
                            reduced_scales=_addr(sc), full_vecs=_addr(arrs["full_vecs"]),
                            entry_ids=_addr(arrs["entry_ids"]),
                            full_vecs_location=FULL_VECS_HOST if full_vecs_host else FULL_VECS_DEVICE,
                            n_clusters=0 if cc is None else cc.shape[0], entry_cluster=_addr(ec),
                            cluster_centroids=_addr(cc))
    h = _P()
    _check(_lib.pilot_index_load(ctypes.byref(desc), ctypes.byref(h)))
    return PilotIndex(h.value)


def load_index_data(idx, full_vecs_host: bool = False) -> PilotIndex:
    """pilot_index_load of an ``index_build.PilotIndexData``."""
    return pilot_index_load(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, idx.full,
                            idx.entry_ids, metric=idx.metric, reduced_dtype=idx.reduced_dtype,
                            reduced_scales=idx.reduced_scales, full_vecs_host=full_vecs_host,
                            entry_cluster=getattr(idx, "entry_cluster", None),
                            cluster_centroids=getattr(idx, "cluster_centroids", None))


def pilot_index_load_files(path: str, flags: int = 0) -> PilotIndex:
    h = _P()
    _check(_lib.pilot_index_load_files(path.encode(), flags, ctypes.byref(h)))
    return PilotIndex(h.value)


def pilot_search(index: PilotIndex, queries, k: int, ef: int, out_ids=None, out_dists=None, stream=None, *,
                 options: pilot_search_options | None = None, counters=None, kernel_ms=None):
    """Top-k search.  ``queries`` is an nq x d float32 numpy array or torch
    tensor (host or CUDA); outputs default to host numpy arrays.  ``stream``
    is a torch.cuda.Stream (or raw handle).  Returns (ids, dists)."""
    nq = int(queries.shape[0])
    if out_ids is None:
        out_ids = np.empty((nq, k), np.int32)
    if out_dists is None:
        out_dists = np.empty((nq, k), np.float32)
    _check_search_buffers(index, queries, k, out_ids, out_dists, counters)
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if options is None and counters is None and kernel_ms is None:
        _check(_lib.pilot_search(index.handle, _addr(queries), nq, k, ef, _addr(out_ids), _addr(out_dists), s))
    else:
        o = options if options is not None else pilot_search_options_default()
        o.counters = _addr(counters)
        o.kernel_ms = _addr(kernel_ms)
        _check(_lib.pilot_search_ex(index.handle, _addr(queries), nq, k, ef, _addr(out_ids), _addr(out_dists), s,
                                    ctypes.byref(o)))
    return out_ids, out_dists


def pilot_search_ex(index: PilotIndex, queries, k: int, ef: int, out_ids=None, out_dists=None, stream=None,
                    options: pilot_search_options | None = None, counters=None, kernel_ms=None):
    """pilot_search with explicit options (``pilot_search_options``).
    ``kernel_ms`` (a float32 numpy array of 3) receives per-kernel device times."""
    return pilot_search(index, queries, k, ef, out_ids, out_dists, stream,
                        options=options if options is not None else pilot_search_options_default(),
                        counters=counters, kernel_ms=kernel_ms)


def pilot_index_info(index: PilotIndex) -> dict:
    return index.info()


def pilot_index_free(index: PilotIndex) -> None:
    index.free()


def pilot_search_noalloc(index: PilotIndex, queries, k: int, ef: int, out_ids, out_dists, stream=None):
    """pilot_search that allocates no device memory during the call: scratch
    comes from a fixed array inside the library.  ``queries``, ``out_ids`` and
    ``out_dists`` must be CUDA tensors (device memory) on one device."""
    _check_search_buffers(index, queries, k, out_ids, out_dists)
    devs = {_device_of(a) for a in (queries, out_ids, out_dists)}
    if None in devs or len(devs) != 1:
        raise ValueError("pilot_search_noalloc needs queries, out_ids and out_dists as CUDA tensors on one device")
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(_lib.pilot_search_noalloc(index.handle, _addr(queries), int(queries.shape[0]), k, ef, _addr(out_ids),
                                     _addr(out_dists), s))
    return out_ids, out_dists


# --------------------------------------------------------------- autotune --

class pilot_tune_result(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("stage_rows", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float)]


_lib.pilot_autotune.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P,
                                ctypes.POINTER(pilot_search_options), ctypes.c_char_p,
                                ctypes.POINTER(pilot_tune_result)]


def pilot_autotune(index: PilotIndex, queries, k: int, ef: int, stream=None, *,
                   options: pilot_search_options | None = None, cache_path: str | None = None) -> dict:
    """Pick the search kernel's launch shape for ``index`` and ef's class by
    timing the caller's queries with the stage switches of ``options`` (see
    include/pilot.h); later searches with automatic options use it.  Returns
    the result fields as a dict."""
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    r = pilot_tune_result()
    _check(_lib.pilot_autotune(index.handle, _addr(queries), int(queries.shape[0]), k, ef, s,
                               ctypes.byref(options) if options is not None else None,
                               cache_path.encode() if cache_path else None, ctypes.byref(r)))
    return {name: getattr(r, name) for name, _ in pilot_tune_result._fields_}


# ---------------------------------------------------------------- serving --

class pilot_serve_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_ef", ctypes.c_int32), ("max_k", ctypes.c_int32),
                ("expansions_per_step", ctypes.c_int32), ("max_new_per_step", ctypes.c_int32),
                ("step_timeout_ms", ctypes.c_int32), ("queue_capacity", ctypes.c_int64),
                ("hbm_budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32)]


class pilot_serve_statistics(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("slots", ctypes.c_int32),
                ("in_flight", ctypes.c_int32), ("queued", ctypes.c_int32), ("visited_overflows", ctypes.c_int32),
                ("qps", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double)]


_lib.pilot_serve_config_default.argtypes = [ctypes.POINTER(pilot_serve_config)]
_lib.pilot_serve_config_default.restype = None
_lib.pilot_serve_create.argtypes = [_P, ctypes.POINTER(pilot_serve_config), ctypes.POINTER(_P)]
_lib.pilot_serve_submit.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
_lib.pilot_serve_submit_batch.argtypes = [_P, _P, ctypes.c_int64, _P, _P, _P]
_lib.pilot_serve_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_int, _P, _P]
_lib.pilot_serve_wait_ex.argtypes = [_P, ctypes.c_uint64, ctypes.c_int, _P, _P, _P]
_lib.pilot_serve_stats.argtypes = [_P, ctypes.POINTER(pilot_serve_statistics)]
_lib.pilot_serve_destroy.argtypes = [_P]
_lib.pilot_serve_destroy.restype = None


def pilot_serve_config_default() -> pilot_serve_config:
    c = pilot_serve_config()
    _lib.pilot_serve_config_default(ctypes.byref(c))
    return c


class PilotServer:
    """Owns a pilot_server handle (continuous-batching search on the GPU)."""

    def __init__(self, handle: int, index: PilotIndex):
        self._h = ctypes.c_void_p(handle)
        self._index = index   # keep the index alive while the server runs

    def submit(self, query, k: int, ef: int) -> int:
        q = np.ascontiguousarray(query, np.float32)
        t = ctypes.c_uint64()
        _check(_lib.pilot_serve_submit(self._h, q.ctypes.data, k, ef, ctypes.byref(t)))
        return t.value

    def submit_batch(self, queries, k, ef) -> np.ndarray:
        """Queue n queries (n x d) with per-query k and ef (arrays or scalars); returns the tickets."""
        q = np.ascontiguousarray(queries, np.float32)
        n = q.shape[0]
        ks = np.ascontiguousarray(np.broadcast_to(np.asarray(k, np.int32), (n,)))
        efs = np.ascontiguousarray(np.broadcast_to(np.asarray(ef, np.int32), (n,)))
        t = np.empty(n, np.uint64)
        _check(_lib.pilot_serve_submit_batch(self._h, q.ctypes.data, n, ks.ctypes.data, efs.ctypes.data,
                                             t.ctypes.data))
        return t

    def wait(self, ticket: int, k: int, timeout_ms: int = 60_000, counters: bool = False):
        """(ids, dists) of a ticket, plus its 8 per-stage counters with ``counters``."""
        ids = np.empty(k, np.int32)
        dists = np.empty(k, np.float32)
        if not counters:
            _check(_lib.pilot_serve_wait(self._h, ticket, timeout_ms, ids.ctypes.data, dists.ctypes.data))
            return ids, dists
        cnt = np.empty(8, np.int32)
        _check(_lib.pilot_serve_wait_ex(self._h, ticket, timeout_ms, ids.ctypes.data, dists.ctypes.data,
                                        cnt.ctypes.data))
        return ids, dists, cnt

    def stats(self) -> dict:
        s = pilot_serve_statistics()
        _check(_lib.pilot_serve_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in pilot_serve_statistics._fields_}

    def destroy(self):
        if self._h:
            _lib.pilot_serve_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pilot_serve_create(index: PilotIndex, config: pilot_serve_config | None = None, **overrides) -> PilotServer:
    c = config if config is not None else pilot_serve_config_default()
    for key, v in overrides.items():
        setattr(c, key, v)
    h = _P()
    _check(_lib.pilot_serve_create(index.handle, ctypes.byref(c), ctypes.byref(h)))
    return PilotServer(h.value, index)


def pilot_serve_submit(server: PilotServer, query, k: int, ef: int) -> int:
    return server.submit(query, k, ef)


def pilot_serve_wait(server: PilotServer, ticket: int, k: int, timeout_ms: int = 60_000):
    return server.wait(ticket, k, timeout_ms)


def pilot_serve_submit_batch(server: PilotServer, queries, k, ef) -> np.ndarray:
    return server.submit_batch(queries, k, ef)


def pilot_serve_wait_ex(server: PilotServer, ticket: int, k: int, timeout_ms: int = 60_000):
    """(ids, dists, counters) of a ticket; counters as pilot_search_options.counters."""
    return server.wait(ticket, k, timeout_ms, counters=True)


def pilot_serve_stats(server: PilotServer) -> dict:
    return server.stats()


def pilot_serve_destroy(server: PilotServer) -> None:
    server.destroy()
