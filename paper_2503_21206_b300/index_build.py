"""Offline index preparation (Sec. 3 / Fig. 2 steps (a)-(c); Sec. 4.1 (1)).

Builds, from a base set X, every input the search reads:

* the full graph (a): the 2R nearest candidates (exact up to 3M rows, from
  inverted lists beyond), the HNSW neighbour-selection heuristic to R, reverse
  edges, re-selection, and a reachability repair from the entry set so that
  every node can be reached;
* the subgraph (b): a seeded uniform node sample, re-connected by the same
  construction among the sampled nodes, stored in the full id space with
  zero-degree rows for unsampled nodes (Sec. 4.3);
* the compact vectors (c): the right singular vectors V of an FP64 SVD of a
  row sample, and the reduced rows x V[:, :d'] of the sampled nodes in FP32,
  BF16 or FP8 E4M3 with per-row FP32 scales;
* a seeded uniform entry set of sampled nodes for fast entry selection.

It also writes / reads the on-disk index format and computes certified exact
ground truth for recall.  This is input generation: it is not timed and holds
none of the search arithmetic.  torch is used for its matrix products (on the
GPU when one is given) and numpy for the FP64 SVD.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import torch

from .synth import Workload

DTYPE_CODES = {"f32": 0, "bf16": 1, "fp8": 2}
IVF_ABOVE = 3_000_000   # graph candidates by inverted lists above this many rows
FILE_MAGIC = "pilot-index 1"


@dataclass
class PilotIndexData:
    """Host arrays of one index (layout of the C-ABI ``pilot_index_desc``)."""
    graph: np.ndarray            # n x R int32, original ids, -1 padded
    subgraph_mask: np.ndarray    # n uint8
    subgraph: np.ndarray         # n x R_sub int32, original ids, -1 padded
    basis: np.ndarray            # d x dp float64
    reduced: np.ndarray          # n_sub x dp: float32 | uint16 (bf16 bits) | uint8 (e4m3 codes)
    reduced_dtype: str           # "f32" | "bf16" | "fp8"
    reduced_scales: np.ndarray | None   # n_sub float32 (fp8)
    full: np.ndarray             # n x d float32 (a CUDA tensor for a base set drawn on the GPU)
    entry_ids: np.ndarray        # n_entry int32
    metric: int                  # 0 L2, 1 IP
    entry_cluster: np.ndarray | None = None       # n_entry int32: coarse cluster of each entry (clustered FES)
    cluster_centroids: np.ndarray | None = None   # n_clusters x dp float32 centroids (reduced space)

    @property
    def n(self):
        return self.full.shape[0]

    @property
    def d(self):
        return self.full.shape[1]

    @property
    def dp(self):
        return self.basis.shape[1]

    def with_reduced(self, dtype: str, reduced_f32: np.ndarray) -> "PilotIndexData":
        """A copy whose reduced rows are ``reduced_f32`` stored as ``dtype``."""
        red, sc = quantize_rows(reduced_f32, dtype)
        return PilotIndexData(self.graph, self.subgraph_mask, self.subgraph, self.basis, red, dtype, sc,
                              self.full, self.entry_ids, self.metric, self.entry_cluster, self.cluster_centroids)


# ------------------------------------------------------------------ kNN --

def _dev(device):
    return torch.device(device if device is not None else "cpu")


def _as_tensor(X, dev):
    """X (numpy array, or a float32 torch tensor already on a device) as an FP32 tensor on dev."""
    if torch.is_tensor(X):
        return X.to(dev, torch.float32)
    return torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)


def _rows(X, idx: np.ndarray) -> np.ndarray:
    """Rows idx of X as a host FP32 array (X numpy or a torch tensor)."""
    if torch.is_tensor(X):
        return X[torch.from_numpy(np.asarray(idx, np.int64)).to(X.device)].float().cpu().numpy()
    return np.asarray(X[idx], np.float32)


def knn_candidates(X: np.ndarray, k: int, device=None, chunk: int = 4096, exclude_self: bool = True):
    """Exact k nearest neighbours of every row of X among the rows of X by
    squared L2 (FP32), ordered by (distance, id).  Returns (ids, dists)."""
    dev = _dev(device)
    Xt = _as_tensor(X, dev)
    n = Xt.shape[0]
    norms = torch.cat([(Xt[r:r + (1 << 20)].double() ** 2).sum(1) for r in range(0, n, 1 << 20)]).float()
    k_eff = min(k, n - 1 if exclude_self else n)
    ids = torch.empty((n, k_eff), dtype=torch.int64, device=dev)
    dst = torch.empty((n, k_eff), dtype=torch.float32, device=dev)
    extra = 8
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        D = norms[s:e, None] - 2.0 * (Xt[s:e] @ Xt.T) + norms[None, :]
        if exclude_self:
            D[torch.arange(e - s, device=dev), torch.arange(s, e, device=dev)] = float("inf")
        kk = min(k_eff + extra, n)
        vals, idx = torch.topk(D, kk, dim=1, largest=False)
        # exact FP32 distances of the candidates, then order by (dist, id)
        diff = Xt[s:e, None, :] - Xt[idx]
        ex = (diff * diff).sum(-1)
        if exclude_self:
            ex = torch.where(idx == torch.arange(s, e, device=dev)[:, None], torch.full_like(ex, float("inf")), ex)
        o1 = torch.argsort(idx, dim=1, stable=True)
        ex, idx = torch.gather(ex, 1, o1), torch.gather(idx, 1, o1)
        o2 = torch.argsort(ex, dim=1, stable=True)
        ex, idx = torch.gather(ex, 1, o2), torch.gather(idx, 1, o2)
        ids[s:e] = idx[:, :k_eff]
        dst[s:e] = ex[:, :k_eff]
    return ids, dst


def ivf_candidates(X: np.ndarray, k: int, device=None, nlist: int | None = None, nprobe: int = 8, seed: int = 0,
                   iters: int = 10, verbose: bool = False):
    """Approximate k nearest neighbours of every row of X among the rows of X
    (squared L2), for base sets too large for the exact quadratic search.

    The rows are split into nlist inverted lists by k-means (a seeded sample,
    Lloyd iterations); the rows of each list are scored (FP32 matrix product)
    against every row of the nprobe lists whose centroids are closest to the
    list's own, the best k + 8 are rescored exactly in FP32, and the first k
    by (distance, id) are kept.  Returns (ids, dists) like knn_candidates; a
    row whose probed lists hold fewer than k others gets -1 / +inf padding."""
    dev = _dev(device)
    Xt = _as_tensor(X, dev)
    n, d = Xt.shape
    if nlist is None:
        nlist = int(min(16384, max(16, n // 2048)))
    nprobe = min(nprobe, nlist)
    rng = np.random.default_rng(seed)
    norms = (Xt * Xt).sum(1)

    def nearest(A, C, Cn, chunk=65536):
        out = torch.empty(A.shape[0], dtype=torch.int64, device=dev)
        for s in range(0, A.shape[0], chunk):
            a = A[s:s + chunk]
            out[s:s + chunk] = torch.argmin(Cn[None, :] - 2.0 * (a @ C.T), dim=1)
        return out

    # k-means on a sample
    samp = torch.from_numpy(np.sort(rng.choice(n, size=min(n, 64 * nlist), replace=False))).to(dev)
    Xs = Xt[samp]
    C = Xs[torch.from_numpy(rng.choice(Xs.shape[0], size=nlist, replace=False)).to(dev)].clone()
    for it in range(iters):
        lab = nearest(Xs, C, (C * C).sum(1))
        cnt = torch.bincount(lab, minlength=nlist).float()
        Cs = torch.zeros_like(C).index_add_(0, lab, Xs)
        ok = cnt > 0
        C[ok] = Cs[ok] / cnt[ok, None]
    labels = nearest(Xt, C, (C * C).sum(1))
    order = torch.argsort(labels, stable=True)
    counts = torch.bincount(labels, minlength=nlist)
    offs = torch.cat([torch.zeros(1, dtype=torch.int64, device=dev), torch.cumsum(counts, 0)]).cpu().numpy()
    Cn = (C * C).sum(1)
    Dcc = Cn[:, None] + Cn[None, :] - 2.0 * (C @ C.T)
    Dcc.fill_diagonal_(-float("inf"))           # each list probes itself first
    probe = torch.topk(Dcc, nprobe, dim=1, largest=False).indices.cpu().numpy()
    order_np = order.cpu().numpy()
    ids = torch.full((n, k), -1, dtype=torch.int64, device=dev)
    dst = torch.full((n, k), float("inf"), dtype=torch.float32, device=dev)
    kk = k + 8
    qchunk = 4096
    for L in range(nlist):
        if offs[L + 1] == offs[L]:
            continue
        q_ids = order[offs[L]:offs[L + 1]]
        pool = torch.cat([order[offs[c]:offs[c + 1]] for c in probe[L]])
        Xp = Xt[pool]
        pn = norms[pool]
        for s in range(0, q_ids.numel(), qchunk):
            qi = q_ids[s:s + qchunk]
            Xq = Xt[qi]
            D = norms[qi][:, None] + pn[None, :] - 2.0 * (Xq @ Xp.T)
            D[torch.arange(qi.numel(), device=dev), torch.arange(s, s + qi.numel(), device=dev)] = float("inf")
            kc = min(kk, pool.numel())
            _, sel = torch.topk(D, kc, dim=1, largest=False)
            cand = pool[sel]
            ex = ((Xq[:, None, :] - Xt[cand]) ** 2).sum(-1)
            ex = torch.where(cand == qi[:, None], torch.full_like(ex, float("inf")), ex)
            o1 = torch.argsort(cand, dim=1, stable=True)
            ex, cand = torch.gather(ex, 1, o1), torch.gather(cand, 1, o1)
            o2 = torch.argsort(ex, dim=1, stable=True)
            ex, cand = torch.gather(ex, 1, o2), torch.gather(cand, 1, o2)
            kt = min(k, kc)
            ok = torch.isfinite(ex[:, :kt])
            ids[qi, :kt] = torch.where(ok, cand[:, :kt], torch.full_like(cand[:, :kt], -1))
            dst[qi, :kt] = ex[:, :kt]
        if verbose and L % 1024 == 0:
            print(f"ivf candidates: list {L}/{nlist}", flush=True)
    return ids, dst


def _pair_dists(Xt, cand):
    """Squared L2 between every pair of candidates of each row: B x C x C."""
    valid = cand >= 0
    V = Xt[cand.clamp(min=0)]
    n2 = (V * V).sum(-1)
    P = n2[:, :, None] + n2[:, None, :] - 2.0 * torch.bmm(V, V.transpose(1, 2))
    P = P.clamp(min=0)
    P[~(valid[:, :, None] & valid[:, None, :])] = float("inf")
    return P


def select_neighbours(Xt: torch.Tensor, node: torch.Tensor, cand: torch.Tensor, dq: torch.Tensor, R: int):
    """HNSW neighbour-selection heuristic, vectorised over rows: walk the
    candidates of each node in (distance, id) order and keep c unless some
    already kept r is closer to c than the node is (dist(c, r) <= dist(c, node)),
    up to R kept.  cand: B x C (-1 = none), dq: B x C distances to the node."""
    B, C = cand.shape
    P = _pair_dists(Xt, cand)
    keep = torch.zeros((B, C), dtype=torch.bool, device=cand.device)
    nk = torch.zeros(B, dtype=torch.int64, device=cand.device)
    for j in range(C):
        ok = (cand[:, j] >= 0) & (cand[:, j] != node) & (nk < R)
        if j > 0:
            viol = (keep[:, :j] & (P[:, j, :j] <= dq[:, j:j + 1])).any(1)
            ok &= ~viol
        keep[:, j] = ok
        nk += ok.long()
    # first R kept, in candidate order
    order = torch.argsort((~keep).to(torch.int8), dim=1, stable=True)[:, :R]
    out = torch.gather(cand, 1, order)
    kept = torch.gather(keep, 1, order)
    return torch.where(kept, out, torch.full_like(out, -1))


def build_graph(X: np.ndarray, R: int, entries_local: np.ndarray, device=None, chunk: int = 0,
                verbose: bool = False, candidates: str = "exact", seed: int = 0) -> np.ndarray:
    """Out-degree-R graph over the rows of X (local ids), -1 padded.
    ``candidates``: "exact" (the 2R nearest) or "ivf" (ivf_candidates, for
    base sets too large for the exact search).  Rows are processed ``chunk``
    at a time (default: as many as keep each chunk's 3R candidate rows near
    8 GB, at least 16384)."""
    dev = _dev(device)
    Xt = _as_tensor(X, dev)
    n = Xt.shape[0]
    if chunk <= 0:
        chunk = int(max(16384, min(65536, 8e9 // (3 * R * Xt.shape[1] * 4))))
    C = min(2 * R, n - 1)
    if candidates == "ivf":
        cand, cd = ivf_candidates(X, C, device=device, seed=seed, verbose=verbose)
    else:
        cand, cd = knn_candidates(X, C, device=device)
    adj = torch.full((n, R), -1, dtype=torch.int64, device=dev)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        adj[s:e] = select_neighbours(Xt, torch.arange(s, e, device=dev), cand[s:e], cd[s:e], R)
    # reverse edges: each node also considers the (up to 2R) closest nodes that
    # selected it, then the union is re-selected to R.
    src = torch.arange(n, device=dev)[:, None].expand(n, R)
    m = adj >= 0
    es, ed = src[m], adj[m]
    edist = torch.empty(es.numel(), dtype=torch.float32, device=dev)
    for a in range(0, es.numel(), 1 << 22):   # in chunks: n x R x d floats would not fit at 10M+ rows
        edist[a:a + (1 << 22)] = ((Xt[es[a:a + (1 << 22)]] - Xt[ed[a:a + (1 << 22)]]) ** 2).sum(-1)
    o = torch.argsort(edist, stable=True)
    es, ed, edist = es[o], ed[o], edist[o]
    o = torch.argsort(ed, stable=True)
    es, ed, edist = es[o], ed[o], edist[o]
    counts = torch.bincount(ed, minlength=n)
    starts = torch.cumsum(counts, 0) - counts
    rank = torch.arange(ed.numel(), device=dev) - starts[ed]
    Rrev = 2 * R
    sel = rank < Rrev
    rev = torch.full((n, Rrev), -1, dtype=torch.int64, device=dev)
    rev[ed[sel], rank[sel]] = es[sel]
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        cand2 = torch.cat([adj[s:e], rev[s:e]], 1)
        cs, _ = torch.sort(cand2, dim=1)
        dup = torch.zeros_like(cs, dtype=torch.bool)
        dup[:, 1:] = cs[:, 1:] == cs[:, :-1]
        cs = torch.where(dup, torch.full_like(cs, -1), cs)
        valid = cs >= 0
        diff = Xt[s:e, None, :] - Xt[cs.clamp(min=0)]
        dq = (diff * diff).sum(-1)
        dq = torch.where(valid, dq, torch.full_like(dq, float("inf")))
        o1 = torch.argsort(torch.where(valid, cs, torch.full_like(cs, n)), dim=1, stable=True)
        cs, dq = torch.gather(cs, 1, o1), torch.gather(dq, 1, o1)
        o2 = torch.argsort(dq, dim=1, stable=True)
        cs, dq = torch.gather(cs, 1, o2), torch.gather(dq, 1, o2)
        adj[s:e] = select_neighbours(Xt, torch.arange(s, e, device=dev), cs, dq, R)
    adj_np = adj.cpu().numpy().astype(np.int32)
    repair_reachability(X, adj_np, entries_local, device=device, verbose=verbose)
    return adj_np


def _reached_from(adj: np.ndarray, sources: np.ndarray) -> np.ndarray:
    """Boolean mask of the nodes reachable from ``sources`` along the edges."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    n, R = adj.shape
    rows = np.repeat(np.arange(n + 1), np.r_[np.full(n, R), [len(sources)]])
    cols = np.concatenate([adj.reshape(-1), sources.astype(np.int32)])
    keep = cols >= 0
    g = sp.csr_matrix((np.ones(int(keep.sum()), np.int8), (rows[keep], cols[keep])), shape=(n + 1, n + 1))
    order = breadth_first_order(g, n, directed=True, return_predecessors=False)
    mask = np.zeros(n + 1, bool)
    mask[order] = True
    return mask[:n]


def repair_reachability(X: np.ndarray, adj: np.ndarray, sources: np.ndarray, device=None,
                        verbose: bool = False, max_rounds: int = 10_000, max_targets: int = 1 << 20) -> int:
    """Make every node reachable from ``sources`` (in place).

    Each round links every unreached node that no other unreached node points
    to (or, if none, the unreached node closest to the reached set -- one per
    weakly connected group of unreached nodes when more than 16 such groups
    remain, so that an index of many separate clusters does not take a round
    per cluster) from its nearest reached node with a free adjacency slot
    (nearest among a seeded sample of max_targets such nodes when there are
    more).
    Returns edges added."""
    dev = _dev(device)
    Xt = _as_tensor(X, dev)
    n, R = adj.shape
    added = 0
    for _ in range(max_rounds):
        reached = _reached_from(adj, sources)
        U = np.nonzero(~reached)[0]
        if U.size == 0:
            return added
        inU = np.zeros(n, bool)
        inU[U] = True
        tgt = adj[U].reshape(-1)
        tgt = tgt[tgt >= 0]
        pointed = np.zeros(n, bool)
        pointed[tgt[inU[tgt]]] = True
        S = U[~pointed[U]]
        free = (adj < 0).any(1) & reached
        F = np.nonzero(free)[0]
        if F.size == 0:
            F = np.nonzero(reached)[0]
        if F.size > max_targets:   # a seeded sample of the candidate targets (large base sets)
            F = np.sort(np.random.default_rng(F.size).choice(F, size=max_targets, replace=False))
        pick = S if S.size else U
        Xs = Xt[torch.from_numpy(pick).to(dev)]
        Xf = Xt[torch.from_numpy(F).to(dev)]
        kk = min(8, F.size)
        best_d = []
        best_i = []
        fn = (Xf ** 2).sum(1)
        for s in range(0, Xs.shape[0], 2048):
            D = (Xs[s:s + 2048] ** 2).sum(1)[:, None] - 2 * Xs[s:s + 2048] @ Xf.T + fn[None, :]
            v, i = torch.topk(D, kk, dim=1, largest=False)
            best_d.append(v.cpu())
            best_i.append(i.cpu())
        bd = torch.cat(best_d).numpy()
        bi = F[torch.cat(best_i).numpy()]
        if not S.size:   # only cycles remain: link the closest node (of each group, when many)
            import scipy.sparse as sp
            from scipy.sparse.csgraph import connected_components
            pos = np.full(n, -1, np.int64)
            pos[U] = np.arange(U.size)
            src = np.repeat(np.arange(U.size), R)
            dst = adj[U].reshape(-1)
            ok = dst >= 0
            ok[ok] = inU[dst[ok]]
            sub = sp.csr_matrix((np.ones(int(ok.sum()), np.int8), (src[ok], pos[dst[ok]])),
                                shape=(U.size, U.size))
            n_comp, label = connected_components(sub, directed=True, connection="weak")
            if n_comp <= 16:
                js = [int(np.argmin(bd[:, 0]))]
            else:
                order = np.lexsort((bd[:, 0], label))          # by group, then distance
                first = np.r_[True, label[order][1:] != label[order][:-1]]
                js = order[first].tolist()
            pick, bd, bi = pick[js], bd[js], bi[js]
        for u, cands in zip(pick, bi):
            placed = False
            for r in cands:
                slots = np.nonzero(adj[r] < 0)[0]
                if slots.size:
                    adj[r, slots[0]] = u
                    placed = True
                    break
            if not placed:          # every candidate is full: overwrite the last slot
                adj[cands[0], R - 1] = u
            added += 1
        if verbose:
            print(f"repair: {U.size} unreached, linked {len(pick)}")
    raise RuntimeError("reachability repair did not converge")


# -------------------------------------------------------------- SVD (c) --

def svd_basis(X: np.ndarray, seed: int, max_rows: int = 262_144) -> np.ndarray:
    """Right singular vectors V (d x d, FP64) of a seeded row sample of X,
    uncentred (Sec. 4.1 (1): X = U Sigma V^T), columns by decreasing singular
    value, each column's largest-magnitude component made positive."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    rows = np.sort(rng.choice(n, size=min(n, max_rows), replace=False))
    A = _rows(X, rows).astype(np.float64)
    _, _, vt = np.linalg.svd(A, full_matrices=False)
    V = vt.T.copy()
    if V.shape[1] < X.shape[1]:   # fewer rows than columns: complete the basis
        q, _ = np.linalg.qr(np.concatenate([V, np.eye(X.shape[1])], 1))
        V = q[:, :X.shape[1]]
    piv = np.argmax(np.abs(V), axis=0)
    V *= np.sign(V[piv, np.arange(V.shape[1])])[None, :]
    return V


def project_rows(X: np.ndarray, basis: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """x V[:, :dp] in FP64, rounded to FP32 (X numpy, or a torch tensor: then on its device)."""
    out = np.empty((X.shape[0], basis.shape[1]), np.float32)
    if torch.is_tensor(X):
        Vt = torch.from_numpy(basis).to(X.device)
        for s in range(0, X.shape[0], chunk):
            out[s:s + chunk] = (X[s:s + chunk].double() @ Vt).float().cpu().numpy()
        return out
    for s in range(0, X.shape[0], chunk):
        out[s:s + chunk] = (X[s:s + chunk].astype(np.float64) @ basis).astype(np.float32)
    return out


def quantize_rows(red: np.ndarray, dtype: str):
    """Store FP32 reduced rows as FP32, BF16 (round to nearest even) or FP8
    E4M3 with scale_r = max|x_r| / 448 (1 for an all-zero row) and codes
    RNE(x / scale) saturated to +-448."""
    if dtype == "f32":
        return np.ascontiguousarray(red, np.float32), None
    t = torch.from_numpy(np.ascontiguousarray(red, np.float32))
    if dtype == "bf16":
        return t.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy(), None
    if dtype == "fp8":
        amax = t.abs().amax(1)
        scale = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
        codes = (t / scale[:, None]).clamp(-448.0, 448.0).to(torch.float8_e4m3fn)
        return codes.view(torch.uint8).numpy().copy(), scale.numpy().astype(np.float32)
    raise ValueError(dtype)


# -------------------------------------------------- entry clusters (Sec. 5) --

def cluster_entries(E: np.ndarray, r: int, seed: int, iters: int = 8):
    """Coarse, bucket-aligned clusters of the entry vectors for the clustered
    FES of Sec. 5: r clusters of ceil(n / r) or fewer entries each.  Seeded
    Lloyd iterations on the reduced FP32 rows, each assignment balanced by
    taking (entry, centroid) pairs in order of distance while the centroid
    has room; centroids are the FP64 means of their members rounded to FP32.
    Returns (cluster of each entry int32, centroids r x dp float32)."""
    E64 = np.asarray(E, np.float64)
    n = E64.shape[0]
    r = max(1, min(r, n))
    rng = np.random.default_rng(seed)
    C = E64[np.sort(rng.choice(n, size=r, replace=False))]
    cap = -(-n // r)
    assign = np.zeros(n, np.int64)
    for _ in range(iters):
        D = (E64 ** 2).sum(1)[:, None] - 2.0 * E64 @ C.T + (C ** 2).sum(1)[None, :]
        order = np.argsort(D, axis=None, kind="stable")
        room = np.full(r, cap)
        assign[:] = -1
        left = n
        for flat in order:
            e, c = divmod(int(flat), r)
            if assign[e] < 0 and room[c] > 0:
                assign[e] = c
                room[c] -= 1
                left -= 1
                if left == 0:
                    break
        for c in range(r):
            m = assign == c
            if m.any():
                C[c] = E64[m].mean(0)
    # keep only non-empty clusters, renumbered in order
    used = np.unique(assign)
    remap = np.full(r, -1, np.int64)
    remap[used] = np.arange(used.size)
    return remap[assign].astype(np.int32), C[used].astype(np.float32)


# ------------------------------------------------------------ the index --

def build_index(X: np.ndarray, R: int, R_sub: int, sample_ratio: float, dp: int, n_entry: int, metric: int,
                seed_graph: int, seed_entry: int, reduced_dtype: str = "f32", device=None,
                verbose: bool = False, keep_reduced_f32: bool = False):
    """Every search input for base set X (see module docstring)."""
    n, d = X.shape
    rng = np.random.default_rng(seed_graph)
    n_sub = max(1, int(round(sample_ratio * n)))
    sampled = np.sort(rng.choice(n, size=n_sub, replace=False)).astype(np.int64)
    erng = np.random.default_rng(seed_entry)
    n_entry = min(n_entry, n_sub)
    entry_local = np.sort(erng.choice(n_sub, size=n_entry, replace=False))
    entry_ids = sampled[entry_local].astype(np.int32)

    # exact candidates up to 3M rows; inverted-list candidates beyond (the
    # exact search is quadratic in n)
    cands = "exact" if n <= IVF_ABOVE else "ivf"
    graph = build_graph(X, R, entry_ids, device=device, verbose=verbose, candidates=cands, seed=seed_graph)
    Xs = X[torch.from_numpy(sampled).to(X.device)] if torch.is_tensor(X) else X[sampled]
    sub_local = build_graph(Xs, R_sub, entry_local, device=device, verbose=verbose,
                            candidates="exact" if n_sub <= IVF_ABOVE else "ivf", seed=seed_graph + 1)
    subgraph = np.full((n, R_sub), -1, np.int32)
    subgraph[sampled] = np.where(sub_local >= 0, sampled[np.maximum(sub_local, 0)], -1).astype(np.int32)
    mask = np.zeros(n, np.uint8)
    mask[sampled] = 1

    V = svd_basis(X, seed_graph)
    basis = np.ascontiguousarray(V[:, :dp])
    red32 = project_rows(Xs, basis)
    del Xs
    red, scales = quantize_rows(red32, reduced_dtype)
    # coarse clusters of the entry set for the clustered FES (r = 32, Sec. 5)
    ent_cluster, centroids = cluster_entries(red32[entry_local], 32, seed_entry)
    full = X if torch.is_tensor(X) else np.ascontiguousarray(X, np.float32)   # a device base set stays there
    idx = PilotIndexData(graph, mask, subgraph, basis, red, reduced_dtype, scales,
                         full, entry_ids, metric, ent_cluster, centroids)
    if keep_reduced_f32:
        return idx, red32, V
    return idx


def build_workload(w: Workload, device=None, n: int | None = None, nq: int | None = None,
                   reduced_dtype: str | None = None, verbose: bool = False):
    """(index, queries, reduced FP32 rows, full basis V) for a workload.  A
    workload marked ``device_base`` (the 25M x 768 one) draws its base set on
    the GPU and keeps it there: ``index.full`` is then a CUDA tensor."""
    from .synth import generate, generate_base_on_device
    if w.extra.get("device_base") and device is not None and str(device).startswith("cuda"):
        X = generate_base_on_device(w, n=n, device=device)
        _, Q = generate(w, n=0, nq=nq)
    else:
        X, Q = generate(w, n=n, nq=nq)
    rd = reduced_dtype or w.reduced_dtypes[0]
    idx, red32, V = build_index(X, w.R, w.R_sub, w.sample_ratio, w.dp, w.n_entry, w.metric, w.graph_seed,
                                w.entry_seed, rd, device=device, verbose=verbose, keep_reduced_f32=True)
    return idx, Q, red32, V


# ------------------------------------------------------------ files --

_FILES = [("graph", "i32"), ("subgraph_mask", "u8"), ("subgraph", "i32"), ("basis", "f64"),
          ("reduced", None), ("reduced_scales", "f32"), ("full", "f32"), ("entry_ids", "i32"),
          ("entry_cluster", "i32"), ("cluster_centroids", "f32")]
_NP = {"i32": np.int32, "u8": np.uint8, "f64": np.float64, "f32": np.float32, "u16": np.uint16}


def checksum64(a: np.ndarray) -> int:
    """Position-weighted word sum: the bytes zero-padded to 8-byte words w_i,
    sum_i w_i * (2i + 1) modulo 2^64.  The C loader computes the same."""
    b = a.tobytes()
    b += b"\0" * (-len(b) % 8)
    w = np.frombuffer(b, dtype="<u8")
    with np.errstate(over="ignore"):
        return int((w * (2 * np.arange(w.size, dtype=np.uint64) + np.uint64(1))).sum(dtype=np.uint64))


def save_index(idx: PilotIndexData, path: str) -> None:
    """Write the directory format read by ``pilot_index_load_files``:
    ``pilot_index.txt`` ("key value" lines) plus one raw little-endian file
    per array.  Each array line carries its byte count."""
    os.makedirs(path, exist_ok=True)
    n, d = idx.full.shape
    lines = [FILE_MAGIC, f"n {n}", f"d {d}", f"dp {idx.dp}", f"R {idx.graph.shape[1]}",
             f"R_sub {idx.subgraph.shape[1]}", f"n_sub {int(idx.subgraph_mask.sum())}",
             f"n_entry {idx.entry_ids.shape[0]}", f"metric {idx.metric}",
             f"reduced_dtype {DTYPE_CODES[idx.reduced_dtype]}"]
    if idx.cluster_centroids is not None:
        lines.append(f"n_clusters {idx.cluster_centroids.shape[0]}")
    for name, kind in _FILES:
        a = getattr(idx, name)
        if a is None:
            continue
        kind = kind or {"f32": "f32", "bf16": "u16", "fp8": "u8"}[idx.reduced_dtype]
        a = np.ascontiguousarray(a, _NP[kind])
        with open(os.path.join(path, name + ".bin"), "wb") as f:
            f.write(a.tobytes())
        lines.append(f"array {name} {kind} {a.nbytes} {checksum64(a):016x}")
    with open(os.path.join(path, "pilot_index.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def load_index(path: str) -> PilotIndexData:
    meta, arrays = {}, {}
    with open(os.path.join(path, "pilot_index.txt")) as f:
        lines = f.read().split("\n")
    assert lines[0] == FILE_MAGIC
    for ln in lines[1:]:
        if not ln:
            continue
        p = ln.split()
        if p[0] == "array":
            arrays[p[1]] = np.fromfile(os.path.join(path, p[1] + ".bin"), dtype=_NP[p[2]])
        else:
            meta[p[0]] = int(p[1])
    n, d, dp = meta["n"], meta["d"], meta["dp"]
    rdt = {v: k for k, v in DTYPE_CODES.items()}[meta["reduced_dtype"]]
    return PilotIndexData(arrays["graph"].reshape(n, meta["R"]), arrays["subgraph_mask"],
                          arrays["subgraph"].reshape(n, meta["R_sub"]), arrays["basis"].reshape(d, dp),
                          arrays["reduced"].reshape(meta["n_sub"], dp), rdt, arrays.get("reduced_scales"),
                          arrays["full"].reshape(n, d), arrays["entry_ids"], meta["metric"],
                          arrays.get("entry_cluster"),
                          arrays["cluster_centroids"].reshape(meta["n_clusters"], dp)
                          if "cluster_centroids" in arrays else None)


# ------------------------------------------------------ ground truth --

def exact_topk(X: np.ndarray, Q: np.ndarray, k: int, metric: int = 0, device=None, margin: int = 32,
               chunk: int = 1024):
    """Exact FP64 top-k ids by (FP64 distance, id) for every query.

    Candidates come from an FP32 matrix product (top k+margin); their distances
    are recomputed in FP64.  A query is certified when the (k+margin)-th FP32
    score, less a bound on the FP32 error, exceeds the k-th FP64 distance;
    uncertified queries are recomputed over all rows in FP64."""
    dev = _dev(device)
    Xt = _as_tensor(X, dev)
    n, d = X.shape
    xn = torch.empty(n, dtype=torch.float64, device=dev)
    for r in range(0, n, 1 << 20):   # FP64 norms in row chunks (a whole FP64 copy may not fit)
        xn[r:r + (1 << 20)] = (Xt[r:r + (1 << 20)].double() ** 2).sum(1)
    kk = min(k + margin, n)
    ids_out = np.empty((Q.shape[0], k), np.int32)
    d_out = np.empty((Q.shape[0], k), np.float64)
    X64 = None if torch.is_tensor(X) or n * d > 50_000_000 else X.astype(np.float64)
    chunk = max(16, min(chunk, int(2_000_000_000 // n)))   # score matrix <= ~8 GB

    def full_fp64(q64):   # every row's FP64 distance, in row chunks on the device
        qt = torch.from_numpy(q64).to(dev)
        out = np.empty(n, np.float64)
        for r in range(0, n, 1 << 20):
            xr = Xt[r:r + (1 << 20)].double()
            out[r:r + xr.shape[0]] = (((xr - qt) ** 2).sum(1) if metric == 0 else -(xr @ qt)).cpu().numpy()
        return out

    for s in range(0, Q.shape[0], chunk):
        Qt = torch.from_numpy(np.ascontiguousarray(Q[s:s + chunk], np.float32)).to(dev)
        ip = Qt @ Xt.T
        if metric == 0:
            qn = (Qt.double() ** 2).sum(1)
            score = (qn[:, None].float() + xn[None, :].float() - 2 * ip)
        else:
            score = -ip
        vals, idx = torch.topk(score, kk, dim=1, largest=False)
        vals, idx = vals.cpu().numpy().astype(np.float64), idx.cpu().numpy()
        q64 = Q[s:s + chunk].astype(np.float64)
        if torch.is_tensor(X):
            xc = Xt[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
        else:
            xc = X[idx].astype(np.float64)
        if metric == 0:
            ex = ((q64[:, None, :] - xc) ** 2).sum(-1)
        else:
            ex = -(q64[:, None, :] * xc).sum(-1)
        qnorm = np.linalg.norm(q64, axis=1)
        xmax = float(np.sqrt(xn.max().item()))
        bound = 4.0 * (d + 2) * 2.0 ** -23 * (qnorm + xmax) ** 2 + 1e-30
        for i in range(ex.shape[0]):
            order = np.lexsort((idx[i], ex[i]))
            top_ids, top_d = idx[i][order][:k], ex[i][order][:k]
            if kk < n and not (vals[i, -1] - bound[i] > top_d[-1]):
                # not certified: exact FP64 over every row
                if X64 is not None:
                    full = ((q64[i] - X64) ** 2).sum(1) if metric == 0 else -(X64 @ q64[i])
                else:
                    full = full_fp64(q64[i])
                o = np.lexsort((np.arange(n), full))[:k]
                top_ids, top_d = o, full[o]
            ids_out[s + i] = top_ids
            d_out[s + i] = top_d
    return ids_out, d_out
