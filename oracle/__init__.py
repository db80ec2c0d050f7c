"""Test infrastructure: ctypes binding to the plain C++ CPU oracle (oracle.cpp).

The oracle restates the PilotANN search (arxiv 2503.21206, Sec. 2.2 Alg. 1,
Sec. 4.1 stages (1)-(3), Sec. 5 dense FES) in FP64 with every distance rounded
once to FP32 (Sec. 6.1).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path never
does and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPE_F32, DTYPE_BF16, DTYPE_FP8 = 0, 1, 2
METRIC_L2, METRIC_IP = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.cpp with plain -O2 (no fast-math, no intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fno-fast-math", "-shared", "-fPIC", "-pthread",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Index(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int64), ("dp", ctypes.c_int64),
                ("R", ctypes.c_int64), ("R_sub", ctypes.c_int64), ("n_entry", ctypes.c_int64),
                ("metric", ctypes.c_int),
                ("graph", ctypes.c_void_p), ("subgraph_mask", ctypes.c_void_p),
                ("subgraph", ctypes.c_void_p), ("basis", ctypes.c_void_p),
                ("reduced", ctypes.c_void_p), ("reduced_dtype", ctypes.c_int),
                ("reduced_scales", ctypes.c_void_p), ("full", ctypes.c_void_p),
                ("entry_ids", ctypes.c_void_p), ("n_clusters", ctypes.c_int64),
                ("entry_cluster", ctypes.c_void_p), ("centroids", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("ef", ctypes.c_int), ("stage1", ctypes.c_int),
                ("stage2_expansions", ctypes.c_int), ("stage3", ctypes.c_int),
                ("use_fes", ctypes.c_int), ("fes_seeds", ctypes.c_int), ("nthreads", ctypes.c_int),
                ("seed_count", ctypes.c_int), ("seed_ids", ctypes.c_void_p)]


class _Outputs(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("dists", ctypes.c_void_p), ("counters", ctypes.c_void_p),
                ("pool1_ids", ctypes.c_void_p), ("pool1_dists", ctypes.c_void_p),
                ("pool2_ids", ctypes.c_void_p), ("pool2_dists", ctypes.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_decode_e4m3.restype = ctypes.c_double
        _lib.oracle_decode_e4m3.argtypes = [ctypes.c_uint8]
        _lib.oracle_decode_bf16.restype = ctypes.c_double
        _lib.oracle_decode_bf16.argtypes = [ctypes.c_uint16]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class OracleIndex:
    """Host arrays of a PilotANN index in the layout the oracle reads.

    graph: n x R int32 (original ids, -1 padded); subgraph_mask: n uint8;
    subgraph: n x R_sub int32 (original ids); basis: d x dp float64;
    reduced: n_sub x dp (float32 | uint16 bf16 bits | uint8 e4m3 codes);
    reduced_scales: n_sub float32 (FP8 only); full: n x d float32;
    entry_ids: int32 original ids; metric 0 = L2, 1 = IP.
    """
    graph: np.ndarray
    subgraph_mask: np.ndarray
    subgraph: np.ndarray
    basis: np.ndarray
    reduced: np.ndarray
    reduced_dtype: int
    reduced_scales: np.ndarray | None
    full: np.ndarray
    entry_ids: np.ndarray
    metric: int = METRIC_L2
    entry_cluster: np.ndarray | None = None     # clustered FES: cluster of each entry
    centroids: np.ndarray | None = None         # n_clusters x dp float32

    def _struct(self):
        arrs = dict(graph=np.ascontiguousarray(self.graph, np.int32),
                    subgraph_mask=np.ascontiguousarray(self.subgraph_mask, np.uint8),
                    subgraph=np.ascontiguousarray(self.subgraph, np.int32),
                    basis=np.ascontiguousarray(self.basis, np.float64),
                    reduced=np.ascontiguousarray(self.reduced),
                    full=np.ascontiguousarray(self.full, np.float32),
                    entry_ids=np.ascontiguousarray(self.entry_ids, np.int32))
        scales = None if self.reduced_scales is None else np.ascontiguousarray(self.reduced_scales, np.float32)
        if self.entry_cluster is not None:
            arrs["entry_cluster"] = np.ascontiguousarray(self.entry_cluster, np.int32)
            arrs["centroids"] = np.ascontiguousarray(self.centroids, np.float32)
        n, d = arrs["full"].shape
        s = _Index(n=n, d=d, dp=arrs["basis"].shape[1], R=arrs["graph"].shape[1],
                   R_sub=arrs["subgraph"].shape[1], n_entry=arrs["entry_ids"].shape[0],
                   metric=self.metric, graph=_ptr(arrs["graph"]), subgraph_mask=_ptr(arrs["subgraph_mask"]),
                   subgraph=_ptr(arrs["subgraph"]), basis=_ptr(arrs["basis"]), reduced=_ptr(arrs["reduced"]),
                   reduced_dtype=self.reduced_dtype, reduced_scales=_ptr(scales), full=_ptr(arrs["full"]),
                   entry_ids=_ptr(arrs["entry_ids"]),
                   n_clusters=0 if self.centroids is None else int(np.asarray(self.centroids).shape[0]),
                   entry_cluster=_ptr(arrs.get("entry_cluster")), centroids=_ptr(arrs.get("centroids")))
        return s, (arrs, scales)


def search(index: OracleIndex, queries: np.ndarray, k: int, ef: int, *, stage1: bool = True,
           stage2_expansions: int = 2, stage3: bool = True, use_fes: bool = True, fes_seeds: int = 1,
           nthreads: int = 1, pools: bool = False, seed_ids: np.ndarray | None = None) -> dict:
    """Staged PilotANN search (Sec. 4.1) of every query; returns a dict of arrays.
    ``fes_seeds`` entries (the best by reduced distance with FES, the first of
    the entry set without) seed stage (1); the paper uses one.  ``use_fes=2``
    is the clustered FES of Sec. 5 (needs the index's entry clusters).  ``seed_ids``
    (nq x T original ids, -1 skipped) instead seeds the final stage alone
    (the experiment of Sec. 4.2); the other stage options are then ignored."""
    lib = _load()
    q = np.ascontiguousarray(queries, np.float32)
    nq = q.shape[0]
    res = dict(ids=np.empty((nq, k), np.int32), dists=np.empty((nq, k), np.float32),
               counters=np.empty((nq, 8), np.int32))
    if pools:
        res.update(pool1_ids=np.empty((nq, ef), np.int32), pool1_dists=np.empty((nq, ef), np.float32),
                   pool2_ids=np.empty((nq, ef), np.int32), pool2_dists=np.empty((nq, ef), np.float32))
    out = _Outputs(**{name: _ptr(res.get(name)) for name, _ in _Outputs._fields_})
    st, keep = index._struct()
    p = _Params(k=k, ef=ef, stage1=int(stage1), stage2_expansions=stage2_expansions, stage3=int(stage3),
                use_fes=int(use_fes), fes_seeds=fes_seeds, nthreads=nthreads)
    seeds = None
    if seed_ids is not None:
        seeds = np.ascontiguousarray(seed_ids, np.int32)
        assert seeds.shape[0] == nq and seeds.ndim == 2
        p.seed_count = seeds.shape[1]
        p.seed_ids = seeds.ctypes.data
    rc = lib.oracle_search(ctypes.byref(st), ctypes.byref(p), _ptr(q), ctypes.c_int64(nq), ctypes.byref(out))
    del seeds
    if rc != 0:
        raise ValueError("oracle_search rejected its arguments")
    del keep
    return res


def project(index: OracleIndex, queries: np.ndarray):
    """q V[:, :dp] in FP64 and its per-component FP32 rounding."""
    lib = _load()
    q = np.ascontiguousarray(queries, np.float32)
    nq, dp = q.shape[0], index.basis.shape[1]
    f64 = np.empty((nq, dp), np.float64)
    f32 = np.empty((nq, dp), np.float32)
    st, keep = index._struct()
    lib.oracle_project(ctypes.byref(st), _ptr(q), ctypes.c_int64(nq), _ptr(f64), _ptr(f32))
    del keep
    return f64, f32


def fes(index: OracleIndex, qproj: np.ndarray):
    """Dense fast entry selection: (entry id, FP32 distance) per projected query."""
    lib = _load()
    q = np.ascontiguousarray(qproj, np.float32)
    nq = q.shape[0]
    ent = np.empty(nq, np.int32)
    dist = np.empty(nq, np.float32)
    st, keep = index._struct()
    lib.oracle_fes(ctypes.byref(st), _ptr(q), ctypes.c_int64(nq), _ptr(ent), _ptr(dist))
    del keep
    return ent, dist


def bruteforce(base: np.ndarray, queries: np.ndarray, k: int, metric: int = METRIC_L2, nthreads: int = 1):
    """Exact FP64 top-k by (distance, id): the recall ground truth."""
    lib = _load()
    b = np.ascontiguousarray(base, np.float32)
    q = np.ascontiguousarray(queries, np.float32)
    nq = q.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    lib.oracle_bruteforce(_ptr(b), ctypes.c_int64(b.shape[0]), ctypes.c_int64(b.shape[1]), ctypes.c_int(metric),
                          _ptr(q), ctypes.c_int64(nq), ctypes.c_int(k), ctypes.c_int(nthreads), _ptr(ids), _ptr(dists))
    return ids, dists


def decode_e4m3(code: int) -> float:
    return _load().oracle_decode_e4m3(code)


def decode_bf16(bits: int) -> float:
    return _load().oracle_decode_bf16(bits)


def recall_at_k(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """recall@k = |retrieved_k ∩ groundtruth_k| / k averaged over queries (Sec. 6.1)."""
    hits = 0
    for f, t in zip(found[:, :k], truth[:, :k]):
        hits += len(set(int(x) for x in f if x >= 0) & set(int(x) for x in t))
    return hits / (k * found.shape[0])
