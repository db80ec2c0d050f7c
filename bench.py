#!/usr/bin/env python3
"""Benchmark of the staged PilotANN search on B300.

One step = one ``pilot_search`` of a whole query batch (every kernel of the
path: projection, FES scoring, fused staged search).  Default workload: the
plain FP32 form, 1,000,000 x 96 unit vectors with a power-law spectrum
(variance ~ i^-0.8) and a seeded rotation, 10,000 queries, R=32, 30% subgraph,
d'=32, k=10, L2.  The ef used is the smallest of the sweep {32, 64, 128, 256}
whose recall@10 against exact FP64 ground truth reaches 0.95; when none does,
the sweep continues with 384 and 512.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead.  Under torchrun each rank holds a
full replica of the index and searches its own batch (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2
EXTRA_EFS = (384, 512)
# the compact precision-form comparison of the default line
FORMS_WORKLOAD, FORMS_N, FORMS_NQ = "c3_powerlaw_2m_d768", 200_000, 2_000


# ----------------------------------------------------------- distributed --

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, device=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda" and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate_throughput(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / max_seconds


# ----------------------------------------------------------------- inputs --

def _cache_dir(name: str, n: int | None, nq_gen: int | None = None) -> str:
    base = os.environ.get("PILOT_BENCH_CACHE", os.path.join(tempfile.gettempdir(), "pilot_bench_cache"))
    return os.path.join(base, f"{name}_n{n or 'full'}" + (f"_q{nq_gen}" if nq_gen else ""))


def load_workload(name: str, n: int | None = None, nq: int | None = None, verbose: bool = True):
    """(workload, index data, queries, exact top-k ids), cached on disk.  The
    query generator is prefix-stable, so ``nq`` takes the first nq queries;
    an ``nq`` above the workload's own query count draws that many (the first
    ones are the workload's queries)."""
    from paper_2503_21206_b300 import synth
    more = nq if nq is not None and nq > synth.WORKLOADS[name].nq else None
    w, idx, Q, gt = _load_full(name, n, verbose, more)
    if nq is not None:
        Q, gt = Q[:nq], gt[:nq]
    return w, idx, np.ascontiguousarray(Q), gt


_BUILT = {}   # in-process cache of workloads too large for the disk cache
DISK_CACHE_MAX_FLOATS = 500_000_000


def _load_full(name: str, n: int | None, verbose: bool, nq_gen: int | None = None):
    import torch
    from paper_2503_21206_b300 import index_build, synth
    w = synth.WORKLOADS[name]
    if (name, n, nq_gen) in _BUILT:
        return _BUILT[(name, n, nq_gen)]
    cdir = _cache_dir(name, n, nq_gen)
    if os.path.exists(os.path.join(cdir, "done")):
        idx = index_build.load_index(cdir)
        return w, idx, np.load(os.path.join(cdir, "queries.npy")), np.load(os.path.join(cdir, "gt.npy"))
    dev = "cuda" if torch.cuda.is_available() else None
    t0 = time.time()
    idx, Q, _, _ = index_build.build_workload(w, device=dev, n=n, nq=nq_gen)
    t1 = time.time()
    gt, _ = index_build.exact_topk(idx.full, Q, w.k, metric=w.metric, device=dev)
    if verbose:
        print(f"[bench] built {name}: index {t1 - t0:.1f}s, ground truth {time.time() - t1:.1f}s", file=sys.stderr)
    if idx.n * idx.d > DISK_CACHE_MAX_FLOATS:   # too large to write out: keep it for this process only
        _BUILT[(name, n, nq_gen)] = (w, idx, Q, gt)
        return w, idx, Q, gt
    os.makedirs(cdir, exist_ok=True)
    index_build.save_index(idx, cdir)
    np.save(os.path.join(cdir, "queries.npy"), Q)
    np.save(os.path.join(cdir, "gt.npy"), gt)
    open(os.path.join(cdir, "done"), "w").write("ok\n")
    return w, idx, Q, gt


def recall_at_k(found, truth, k):
    hits = 0
    for f, t in zip(found[:, :k], truth[:, :k]):
        hits += len(set(f.tolist()) & set(t.tolist()))
    return hits / (k * len(found))


# -------------------------------------------------------------- helpers --

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.path = gpu_index, None, None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            self.proc.wait(timeout=10)

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(float(r[1]) for r in rows),
                "sm_max_mhz": max(float(r[2]) for r in rows), "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows)}


def algorithmic_bytes(counters: np.ndarray, k: int, idx, T: int = 8) -> float:
    """Bytes the method must move for one batch, from per-query counters:
    stage (1): exp1 * 4 R_sub + dist1 * (d' b + s); re-rank: n_rerank * 4 d;
    stage (2): exp2 * 4 R_sub + dist2 * 4 d; stage (3): exp3 * 4 R + dist3 * 4 d;
    FES check T (d' b + s); the query (4 d), its projection (4 d') and the output (8 k).
    b = bytes per reduced element, s = 4 for the FP8 per-row scale."""
    b = {"f32": 4, "bf16": 2, "fp8": 1}[idx.reduced_dtype]
    s = 4 if idx.reduced_dtype == "fp8" else 0
    d, dp, R, Rs = idx.d, idx.dp, idx.graph.shape[1], idx.subgraph.shape[1]
    c = counters.astype(np.float64)
    per_q = (c[:, 0] * 4 * Rs + c[:, 1] * (dp * b + s) + c[:, 6] * 4 * d + c[:, 2] * 4 * Rs + c[:, 3] * 4 * d +
             c[:, 4] * 4 * R + c[:, 5] * 4 * d + T * (dp * b + s) + 4 * d + 4 * dp + 8 * k)
    return float(per_q.sum())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("search_impl.cuh", "device_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2503_21206_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, ef: int, nq: int):
    """DRAM bytes per launch of the search kernel from the committed ncu summary
    (profiles/search_kernel_traffic.json), scaled to nq queries; None when it
    was taken on another kernel source, workload or ef."""
    p = os.path.join(ROOT, "profiles", "search_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_hash") != kernel_source_hash() or d.get("workload") != workload or d.get("ef") != ef:
        return None
    return float(d["dram_bytes_per_query"]) * nq


def oracle_index(idx):
    import oracle
    return oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced,
                              {"f32": 0, "bf16": 1, "fp8": 2}[idx.reduced_dtype], idx.reduced_scales, idx.full,
                              idx.entry_ids, idx.metric)


def oracle_sample(idx, Q, k, ef, budget_s: float = 12.0, min_q: int = 64, max_q: int = 4000, threads: int = 0):
    """The oracle as it stands, on `threads` host threads (all cores by
    default), over a bounded query sample.  Returns (qps, queries, seconds,
    threads)."""
    import oracle
    oi = oracle_index(idx)
    threads = threads or os.cpu_count() or 1
    n = min(min_q, len(Q))
    t0 = time.perf_counter()
    oracle.search(oi, Q[:n], k, ef, nthreads=threads)
    dt = time.perf_counter() - t0
    if dt < budget_s / 4 and n < len(Q):
        n = int(min(max_q, len(Q), max(n, n * budget_s / max(dt, 1e-3))))
        t0 = time.perf_counter()
        oracle.search(oi, Q[:n], k, ef, nthreads=threads)
        dt = time.perf_counter() - t0
    return n / dt, n, dt, threads


def cpu_baseline_entry(idx, Q, k, ef) -> dict:
    """The oracle on all host cores (the reported value) and on one thread."""
    qps, ns, secs, threads = oracle_sample(idx, Q, k, ef)
    qps1, ns1, secs1, _ = oracle_sample(idx, Q, k, ef, budget_s=4.0, min_q=8, max_q=512, threads=1)
    return {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"first {ns} of {len(Q)} queries, ef={ef}, {secs:.1f}s on {threads} host threads",
            "value_1thread": qps1,
            "sample_1thread": f"first {ns1} of {len(Q)} queries, ef={ef}, {secs1:.1f}s on 1 host thread"}


# ------------------------------------------------------------------ arms --

def serving_run(pilot, g, Q, gt, rate: float, n_req: int, seed: int = 5, fixed_ef: int = 0, ef_set=None,
                **cfg) -> dict:
    """Poisson arrivals at `rate` requests/s of n_req requests with k drawn
    from {1, 10, 100} and ef uniform in 32..512 (ef >= k) -- or, with
    `fixed_ef`, k = 10 and that ef for all; with `ef_set`, k = 10 and ef drawn
    from the set -- submitted from this thread as their arrival times pass;
    returns the server's statistics and recall@min(k, 10) of the answers."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    if fixed_ef:
        ks = np.full(n_req, 10)
        efs = np.full(n_req, fixed_ef)
    elif ef_set:
        ks = np.full(n_req, 10)
        efs = rng.choice(np.asarray(ef_set), size=n_req)
    else:
        ks = rng.choice([1, 10, 100], size=n_req)
        efs = np.array([int(rng.integers(max(32, k), 513)) for k in ks])
    rows = rng.integers(0, len(Q), n_req)
    Qr = np.ascontiguousarray(Q[rows])
    srv = pilot.pilot_serve_create(g, **cfg)
    tickets = []
    try:
        # every request whose arrival time has passed goes in with one call
        t0 = time.perf_counter()
        i = 0
        while i < n_req:
            now = time.perf_counter() - t0
            j = int(np.searchsorted(arrivals, now, side="right"))
            if j > i:
                tickets.extend(srv.submit_batch(Qr[i:j], ks[i:j], efs[i:j]).tolist())
                i = j
            if i < n_req:
                time.sleep(max(0.0, min(1e-4, arrivals[i] - now)))
        hits = tot = 0
        for j, t in enumerate(tickets):
            ids, _ = srv.wait(t, int(ks[j]))
            kk = min(int(ks[j]), 10)
            hits += len(set(ids[:kk].tolist()) & set(gt[rows[j], :kk].tolist()))
            tot += kk
        st = srv.stats()
    finally:
        srv.destroy()
    return {"offered_rate": rate, "requests": n_req, "qps": round(st["qps"], 1), "p50_ms": round(st["p50_ms"], 3),
            "p99_ms": round(st["p99_ms"], 3), "mean_ms": round(st["mean_ms"], 3), "slots": st["slots"],
            "steps": st["steps"], "recall@min(k,10)": round(hits / tot, 5), "mean_ef": float(efs.mean()),
            "k_mix": "10" if (fixed_ef or ef_set) else "1/10/100 uniform",
            "ef_mix": (f"{fixed_ef} for all" if fixed_ef else
                       (f"uniform over {sorted(int(e) for e in ef_set)}" if ef_set else "uniform 32..512, ef >= k"))}


def run_reference(args):
    """The oracle as the reference arm: same workload, metric and ef rule."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq)
    threads = os.cpu_count() or 1
    oi = oracle_index(idx)
    ef = args.ef
    if not ef:   # the GPU arm's rule, judged on a 256-query sample
        ns = min(256, len(Q))
        for cand in list(w.efs) + [e for e in EXTRA_EFS if e > max(w.efs)]:
            ef = cand
            r = oracle.search(oi, Q[:ns], w.k, cand, nthreads=threads)
            if recall_at_k(r["ids"], gt[:ns], w.k) >= 0.95:
                break
    qps0, _, _, _ = oracle_sample(idx, Q, w.k, ef, budget_s=2.0, min_q=32, max_q=256)
    per_step = int(max(16, min(len(Q), qps0 * 8.0)))
    for _ in range(args.warmup):
        oracle.search(oi, Q[:16], w.k, ef, nthreads=threads)
    times, hits = [], []
    for s in range(args.steps):
        lo = (s * per_step) % max(1, len(Q) - per_step + 1)
        t0 = time.perf_counter()
        r = oracle.search(oi, Q[lo:lo + per_step], w.k, ef, nthreads=threads)
        times.append(time.perf_counter() - t0)
        hits.append(recall_at_k(r["ids"], gt[lo:lo + per_step], w.k))
    total = sum(times)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": "QPS@recall10=0.95", "value": value, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 accumulate, f32-rounded distances", "data": "synthetic",
            "config": {"workload": args.workload, "n": idx.n, "d": idx.d, "nq": len(Q), "k": w.k, "ef": ef,
                       "recall@10": round(float(np.mean(hits)), 5), "l2": "n/a (host cores)"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} of {len(Q)} queries per step, ef={ef}, {threads} threads"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def distance_error(idx, Q, ids, dists) -> float:
    """Largest relative error of the returned distances against the FP64
    distances of the same ids (the FP64 brute-force definition)."""
    worst = 0.0
    for s in range(0, len(Q), 1024):
        I = ids[s:s + 1024].astype(np.int64)
        ok = I >= 0
        X = idx.full[np.where(ok, I, 0)].astype(np.float64)
        q = Q[s:s + 1024, None, :].astype(np.float64)
        ref = ((X - q) ** 2).sum(-1) if idx.metric == 0 else -(X * q).sum(-1)
        err = np.abs(dists[s:s + 1024].astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-30)
        worst = max(worst, float(err[ok].max()) if ok.any() else 0.0)
    return worst


def timed_steps(search, stream, flush, steps: int, warmup: int, kms):
    """(mean step ms, mean search-kernel ms) over `steps` device-timed calls,
    L2 flushed before each."""
    import torch
    for _ in range(warmup):
        search()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    step_ms, search_ms = [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev0.record(stream)
        search()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        search_ms.append(float(kms[2]))
    return statistics.mean(step_ms), statistics.mean(search_ms)


def measure_forms(workload, n, nq, steps, warmup, serve_requests, serve_budget, autotune, fixed_ef=0,
                  serving=True, dtypes=None, plain=True, log=True):
    """Precision forms of one workload on one GPU: reduced rows in FP32, BF16
    and FP8-E4M3 (the workload's list, or `dtypes`), plus the plain form (only
    the final stage: Algorithm 1 on the full graph with full rows, seeded by
    FES).  For each, the smallest swept ef reaching recall@10 >= 0.95 against
    the FP64 brute force, batch QPS there, the search kernel's fraction of HBM
    peak, the distance error against FP64, and a saturating serving run at
    that ef (offered at twice the batch rate).  Returns (index, list of
    per-form records)."""
    import torch
    from paper_2503_21206_b300 import pilot
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w, idx32, Q, gt = load_workload(workload, n, nq)
    if idx32.reduced_dtype != "f32":
        raise SystemExit("the precision forms need a workload whose index stores FP32 reduced rows")
    red32 = idx32.reduced
    nq, k = len(Q), w.k
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    cnt = torch.empty((nq, 8), dtype=torch.int32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    kms = np.zeros(3, np.float32)
    peak, peak_kind = measured_peaks()
    efs = [fixed_ef] if fixed_ef else list(w.efs) + [e for e in EXTRA_EFS if e > max(w.efs)]
    forms = [(dt, dict()) for dt in (dtypes or w.reduced_dtypes)]
    if plain:
        forms.append(("f32", dict(stage1=0, stage2_expansions=0)))
    out = []
    for dt, sw in forms:
        idx = idx32 if dt == "f32" else idx32.with_reduced(dt, red32)
        g = pilot.load_index_data(idx)
        opts = pilot.pilot_search_options_default()
        for key, v in sw.items():
            setattr(opts, key, v)

        def search(ef, counters=None):
            return pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, options=opts, counters=counters,
                                         kernel_ms=kms)

        search(efs[0])   # untimed: module loading and the first workspace allocation
        torch.cuda.synchronize()
        sweep, ef = [], None
        for cand in efs:
            search(cand)
            torch.cuda.synchronize()
            rec = recall_at_k(ids.cpu().numpy(), gt, k)
            sweep.append({"ef": cand, "recall@10": round(rec, 5), "search_ms": round(float(kms[2]), 3)})
            ef = cand
            if rec >= 0.95:
                break
        tuned = pilot.pilot_autotune(g, qd, k, ef, stream, options=opts) if autotune else None
        search(ef, cnt)
        torch.cuda.synchronize()
        counters = cnt.cpu().numpy()
        h_ids, h_d = ids.cpu().numpy(), dists.cpu().numpy()
        recall = recall_at_k(h_ids, gt, k)
        step_ms, search_ms = timed_steps(lambda: search(ef), stream, flush, steps, warmup, kms)
        alg = algorithmic_bytes(counters, k, idx)
        c = counters.astype(np.float64)
        rec_form = {"form": "plain (final stage only)" if sw else "staged", "reduced_dtype": dt, "ef": ef,
                    "recall@10": round(recall, 5), "qps": nq / (step_ms / 1000.0), "ms_per_batch": step_ms,
                    "search_kernel_ms": search_ms, "hbm_gbs": alg / (search_ms / 1000.0) / 1e9,
                    "hbm_frac": alg / (search_ms / 1000.0) / 1e9 / peak,
                    "max_rel_dist_err_vs_fp64": distance_error(idx, Q, h_ids, h_d), "sweep": sweep,
                    "autotuned": tuned,
                    "mean_counters": {name: round(float(c[:, i].mean()), 1) for i, name in
                                      enumerate(["exp1", "dist1", "exp2", "dist2", "exp3", "dist3", "rerank"])}}
        if serving and not sw:   # the server always runs every stage
            rate = 2.0 * rec_form["qps"]
            rec_form["serving"] = serving_run(pilot, g, Q, gt, rate, min(serve_requests, int(rate * 4) + 1000),
                                              fixed_ef=ef, max_ef=512, max_k=100,
                                              expansions_per_step=serve_budget)
        out.append(rec_form)
        if log:
            print(json.dumps(rec_form), file=sys.stderr, flush=True)
        g.free()
        del g
    return idx32, out


def run_forms(args):
    """The precision forms of --workload as one JSON line (see measure_forms)."""
    idx32, out = measure_forms(args.workload, args.n, args.nq, args.steps, args.warmup, args.serve_requests,
                               args.serve_budget, not args.no_autotune, fixed_ef=args.ef,
                               serving=not args.no_serving)
    peak, peak_kind = measured_peaks()
    base = next(f for f in out if f["form"] != "staged")
    from paper_2503_21206_b300 import synth
    w = synth.WORKLOADS[args.workload]
    line = {"metric": "QPS@recall10=0.95 by precision form", "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
            "config": {"workload": args.workload, "n": idx32.n, "d": idx32.d, "dp": idx32.dp,
                       "nq": args.nq or w.nq, "k": w.k, "metric": "ip" if idx32.metric else "l2",
                       "R": int(idx32.graph.shape[1]),
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"},
            "peak": {"hbm_gbs": peak, "source": peak_kind},
            "forms": out,
            "qps_vs_plain": {f["reduced_dtype"] + ("" if f["form"] == "staged" else "_plain"):
                             round(f["qps"] / base["qps"], 3) for f in out}}
    print(json.dumps(line), flush=True)
    return 0


def forms_summary(args) -> dict:
    """The compact comparison in the default line: on the first FORMS_N rows
    of the 768-d power-law workload (IP, d' = 128, where BF16 rows are half
    the bytes of FP32 ones), the served BF16 staged form against the served
    FP32 staged form and the plain FP32 form, each at its smallest ef reaching
    recall@10 >= 0.95, measured in this run."""
    idx32, out = measure_forms(FORMS_WORKLOAD, FORMS_N, FORMS_NQ, 3, 3, 30_000, args.serve_budget,
                               autotune=False, dtypes=("f32", "bf16"), log=False)
    by = {("plain" if f["form"] != "staged" else f["reduced_dtype"]): f for f in out}
    brief = {}
    for name, f in by.items():
        e = {"ef": f["ef"], "recall@10": f["recall@10"], "batch_qps": round(f["qps"], 1),
             "hbm_frac": round(f["hbm_frac"], 4)}
        if "serving" in f:
            e["served_qps"] = f["serving"]["qps"]
            e["served_recall@min(k,10)"] = f["serving"]["recall@min(k,10)"]
            e["served_p99_ms"] = f["serving"]["p99_ms"]
        brief[name] = e
    res = {"workload": f"{FORMS_WORKLOAD} first {idx32.n} rows, {FORMS_NQ} queries", "forms": brief}
    if "served_qps" in brief.get("bf16", {}) and "served_qps" in brief.get("f32", {}):
        res["served_bf16_over_served_f32"] = round(brief["bf16"]["served_qps"] / brief["f32"]["served_qps"], 3)
    if "served_qps" in brief.get("bf16", {}) and "plain" in brief:
        res["served_bf16_over_plain_f32_batch"] = round(brief["bf16"]["served_qps"] / brief["plain"]["batch_qps"], 3)
    return res


def run_memory_bounded(args):
    """The memory-bounded configuration: full vectors in pinned host memory,
    read over the host link by the re-rank and stages (2)(3); the GPU holds
    the graphs, the subgraph's reduced rows and the entries.  Batch operating
    points over the workload's ef list (recall@10 against FP64 brute force,
    QPS, host-link GB/s of full-row bytes), the QPS at the smallest ef
    reaching recall 0.9 and 0.95, and a Poisson serving run with mixed ef."""
    import torch
    from paper_2503_21206_b300 import pilot
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    t0 = time.time()
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq)
    t_build = time.time() - t0
    t0 = time.time()
    g = pilot.load_index_data(idx, full_vecs_host=True)
    t_load = time.time() - t0
    info = g.info()
    nq, k = len(Q), w.k
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    cnt = torch.empty((nq, 8), dtype=torch.int32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    kms = np.zeros(3, np.float32)
    d_pad = (idx.d + 31) // 32 * 32
    batch = []
    for ef in list(w.efs):
        pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, counters=cnt, kernel_ms=kms)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt, k)
        c = cnt.cpu().numpy().astype(np.float64)
        host_bytes = float((c[:, 6] + c[:, 3] + c[:, 5]).sum()) * d_pad * 4   # full rows read over the host link
        step_ms, search_ms = timed_steps(lambda: pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream,
                                                                       kernel_ms=kms),
                                         stream, flush, args.steps, args.warmup, kms)
        batch.append({"ef": ef, "recall@10": round(rec, 5), "qps": nq / (step_ms / 1000.0),
                      "search_kernel_ms": search_ms, "host_link_gbs": host_bytes / (search_ms / 1000.0) / 1e9,
                      "mean_counters": {nm: round(float(c[:, i].mean()), 1) for i, nm in
                                        enumerate(["exp1", "dist1", "exp2", "dist2", "exp3", "dist3", "rerank"])}})
        print(json.dumps(batch[-1]), file=sys.stderr, flush=True)
    # the same index with the full vectors in device memory, for comparison
    g_dev = pilot.load_index_data(idx)
    for b in batch:
        step_ms, search_ms = timed_steps(lambda: pilot.pilot_search_ex(g_dev, qd, k, b["ef"], ids, dists, stream,
                                                                       kernel_ms=kms),
                                         stream, flush, args.steps, args.warmup, kms)
        b["device_resident_qps"] = nq / (step_ms / 1000.0)
    g_dev.free()
    at = {}
    for target in (0.9, 0.95):
        hit = next((b for b in batch if b["recall@10"] >= target), None)
        at[str(target)] = None if hit is None else {"ef": hit["ef"], "qps": round(hit["qps"], 1),
                                                     "recall@10": hit["recall@10"],
                                                     "device_resident_qps": round(hit["device_resident_qps"], 1)}
    best = max(batch, key=lambda b: b["recall@10"])
    at["max_recall"] = {"ef": best["ef"], "qps": round(best["qps"], 1), "recall@10": best["recall@10"]}
    ef_set = [e for e in (128, 256) if e in w.efs] or list(w.efs[:2])
    base_qps = min(b["qps"] for b in batch if b["ef"] in ef_set)
    rate = 0.6 * base_qps
    serving = serving_run(pilot, g, Q, gt, rate, int(min(args.serve_requests, max(2000, rate * 6))), ef_set=ef_set,
                          max_ef=max(ef_set), max_k=k, expansions_per_step=args.serve_budget)
    line = {"metric": "memory-bounded: QPS at recall@10 0.9 / 0.95 and p99", "unit": "queries/s", "n_gpus": 1,
            "data": "synthetic", "config": {"workload": args.workload, "n": idx.n, "d": idx.d, "dp": idx.dp,
                                            "reduced_dtype": idx.reduced_dtype, "nq": nq, "k": k,
                                            "metric": "ip" if idx.metric else "l2",
                                            "full_vecs": "pinned host memory, read over the host link",
                                            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"},
            "device_bytes_of_index": info["device_bytes"], "host_bytes_of_full_vectors": int(idx.n) * d_pad * 4,
            "build_s": round(t_build, 1), "load_s": round(t_load, 1),
            "qps_at_recall": at, "batch": batch, "serving": serving}
    print(json.dumps(line), flush=True)
    return 0


def run_serve_sweep(args):
    """The serving configuration: Poisson arrivals of mixed k in {1, 10, 100}
    and ef in 32..512 at several offered rates, p50/p99 latency and served
    QPS at each, beside the batch operating point of the same index."""
    import torch
    from paper_2503_21206_b300 import pilot
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq)
    g = pilot.load_index_data(idx)
    nq, k = len(Q), w.k
    rates = [float(r) for r in args.serve_rates.split(",")]
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    kms = np.zeros(3, np.float32)
    batch = []
    for ef in (64, 128, 256, 512):
        pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, kernel_ms=kms)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt, k)
        step_ms, search_ms = timed_steps(lambda: pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream,
                                                                       kernel_ms=kms),
                                         stream, flush, args.steps, args.warmup, kms)
        batch.append({"ef": ef, "recall@10": round(rec, 5), "qps": nq / (step_ms / 1000.0)})
    rows = []
    for rate in rates:
        r = serving_run(pilot, g, Q, gt, rate, min(int(rate * 2.0), args.serve_requests), max_ef=512, max_k=100,
                        expansions_per_step=args.serve_budget)
        rows.append(r)
        print(json.dumps(r), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "serving p50/p99 and QPS by offered rate", "workload": args.workload, "n": idx.n,
                      "d": idx.d, "dp": idx.dp, "reduced_dtype": idx.reduced_dtype, "nq": nq,
                      "data": "synthetic", "budget": args.serve_budget, "batch": batch, "serving": rows}),
          flush=True)
    return 0


def run_sweep_sub(args):
    """The GPU-piloting sensitivity of the paper's appendix (sampling ratio x
    SVD ratio d'/d) on synthetic data: for each pair, the staged search's
    smallest swept ef reaching recall@10 >= 0.95 and its batch QPS, beside
    the plain final-stage form.  The full graph, the queries and the ground
    truth are the workload's; only the subgraph (sample, re-built graph,
    entries) and the reduced rows change per cell."""
    import torch
    from paper_2503_21206_b300 import index_build, pilot
    from paper_2503_21206_b300.index_build import PilotIndexData
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq)
    X, n, d = idx.full, idx.n, idx.d
    nq, k = len(Q), w.k
    V = index_build.svd_basis(X, w.graph_seed)
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    kms = np.zeros(3, np.float32)
    efs = list(w.efs) + [e for e in EXTRA_EFS if e > max(w.efs)]

    def operating_point(g, opts):
        ef_hit, rec = None, 0.0
        for ef in efs:
            pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, options=opts, kernel_ms=kms)
            torch.cuda.synchronize()
            rec = recall_at_k(ids.cpu().numpy(), gt, k)
            ef_hit = ef
            if rec >= 0.95:
                break
        step_ms, _ = timed_steps(lambda: pilot.pilot_search_ex(g, qd, k, ef_hit, ids, dists, stream,
                                                               options=opts, kernel_ms=kms),
                                 stream, flush, args.steps, args.warmup, kms)
        return {"ef": ef_hit, "recall@10": round(rec, 5), "qps": nq / (step_ms / 1000.0)}

    g = pilot.load_index_data(idx)
    plain = pilot.pilot_search_options_default()
    plain.stage1, plain.stage2_expansions = 0, 0
    base_plain = operating_point(g, plain)
    g.free()
    cells = []
    for sr in [float(x) for x in args.sample_ratios.split(",")]:
        rng = np.random.default_rng(w.graph_seed)
        n_sub = max(1, int(round(sr * n)))
        sampled = np.sort(rng.choice(n, size=n_sub, replace=False)).astype(np.int64)
        erng = np.random.default_rng(w.entry_seed)
        n_entry = min(w.n_entry, n_sub)
        entry_local = np.sort(erng.choice(n_sub, size=n_entry, replace=False))
        sub_local = index_build.build_graph(X[sampled], w.R_sub, entry_local, device="cuda")
        subgraph = np.full((n, w.R_sub), -1, np.int32)
        subgraph[sampled] = np.where(sub_local >= 0, sampled[np.maximum(sub_local, 0)], -1).astype(np.int32)
        mask = np.zeros(n, np.uint8)
        mask[sampled] = 1
        for svd_ratio in [float(x) for x in args.svd_ratios.split(",")]:
            dp = max(1, int(round(svd_ratio * d)))
            if dp > 128:   # the library keeps d' <= 128
                cells.append({"sample_ratio": sr, "svd_ratio": svd_ratio, "dp": dp,
                              "skipped": "d' above the library's limit of 128"})
                continue
            basis = np.ascontiguousarray(V[:, :dp])
            red = index_build.project_rows(X[sampled], basis)
            cell_idx = PilotIndexData(idx.graph, mask, subgraph, basis, red, "f32", None, X,
                                      sampled[entry_local].astype(np.int32), idx.metric)
            g = pilot.load_index_data(cell_idx)
            op = operating_point(g, pilot.pilot_search_options_default())
            g.free()
            op.update({"sample_ratio": sr, "svd_ratio": svd_ratio, "dp": dp,
                       "qps_vs_plain": round(op["qps"] / base_plain["qps"], 3)})
            cells.append(op)
            print(json.dumps(op), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "QPS@recall10=0.95 by sampling ratio x SVD ratio", "workload": args.workload,
                      "n": n, "d": d, "nq": nq, "plain_final_stage": base_plain, "cells": cells,
                      "data": "synthetic"}), flush=True)
    return 0


def run_gather_ceiling(args):
    """Random-row read bandwidth of this GPU for the row sizes the search
    kernel reads (32 B visited buckets, 128 B adjacency rows, full and
    reduced rows): torch.embedding_bag sums bags of 64 random rows of a
    4 GB table, so nearly all DRAM traffic is the random reads.  A ceiling
    for the search kernel's access pattern beside the streaming copy peak;
    the library's kernels play no part in it."""
    import torch
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    table_bytes, gathered, bag = 4 << 30, 2 << 30, 64
    out = []
    for row_bytes in (32, 128, 384, 3072):
        n_rows = table_bytes // row_bytes
        table = torch.ones((n_rows, row_bytes // 4), dtype=torch.float32, device=device)
        m = gathered // row_bytes // bag * bag
        idx = torch.randint(0, n_rows, (m,), device=device, generator=torch.Generator(device).manual_seed(1))
        offs = torch.arange(0, m, bag, device=device)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for rep in range(args.warmup + args.steps):
            ev0.record()
            torch.nn.functional.embedding_bag(idx, table, offs, mode="sum")
            ev1.record()
            ev1.synchronize()
            if rep >= args.warmup:
                ts.append(ev0.elapsed_time(ev1) / 1000.0)
        t = statistics.median(ts)
        out.append({"row_bytes": row_bytes, "rows": m, "random_read_gbs": round(m * row_bytes / t / 1e9, 1),
                    "ms": round(t * 1000, 3)})
        del table, idx, offs
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "random-row read bandwidth", "unit": "GB/s", "method": "torch embedding_bag, "
                      f"sum over bags of {bag} random rows of a 4 GB table", "rows": out}), flush=True)
    return 0


def run_tau(args):
    """The analysis of Sec. 4.2 (its tau/ef figures) on synthetic data: the
    final stage alone (Algorithm 1 on the full graph with full vectors),
    its candidate list of size ef seeded with tau true neighbours plus
    ef - tau random nodes.  For each tau/ef and ef: recall@10 and the
    distance calculations per query (seeds scored + new distances).  Then
    the calculations needed for recall@10 = 0.9 (interpolated over ef), the
    saving against tau = 0, and the acceleration threshold: the smallest
    tau/ef with a 2x saving."""
    import torch
    from paper_2503_21206_b300 import index_build, pilot
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w, idx, Q, gt10 = load_workload(args.workload, args.n, args.nq)
    Q = Q[: min(len(Q), 2000)]
    gt10 = gt10[: len(Q)]
    nq, k = len(Q), w.k
    efs = (32, 64, 128, 256, 512)
    fracs = (0.0, 1 / 16, 1 / 8, 3 / 16, 1 / 4)
    gt, _ = index_build.exact_topk(idx.full, Q, int(max(efs) * max(fracs)), metric=idx.metric, device="cuda")
    g = pilot.load_index_data(idx)
    rng = np.random.default_rng(7)
    curves = []
    for f in fracs:
        pts = []
        for ef in efs:
            tau = int(round(f * ef))
            seeds = np.empty((nq, ef), np.int32)
            for i in range(nq):
                known = gt[i, :tau]
                cand = rng.choice(idx.n, size=ef + tau, replace=False)
                rest = cand[~np.isin(cand, known)][: ef - tau]
                seeds[i, :tau] = known
                seeds[i, tau:] = rest
            o = pilot.pilot_search_options_default()
            o.stage1, o.stage2_expansions = 0, 0
            o.seed_ids, o.seed_count = seeds.ctypes.data, ef
            cnt = np.empty((nq, 8), np.int32)
            ids, _ = pilot.pilot_search_ex(g, Q, k, ef, options=o, counters=cnt)
            calcs = float((cnt[:, 5] + cnt[:, 6]).mean())
            pts.append({"ef": ef, "tau": tau, "recall@10": round(recall_at_k(ids, gt10, k), 5),
                        "calcs_per_query": round(calcs, 1), "expansions": round(float(cnt[:, 4].mean()), 1)})
        curves.append({"tau_over_ef": f, "points": pts})
        print(json.dumps(curves[-1]), file=sys.stderr, flush=True)

    def calcs_at(points, target):
        xs = [p["recall@10"] for p in points]
        ys = [p["calcs_per_query"] for p in points]
        for j in range(1, len(xs)):
            if xs[j - 1] < target <= xs[j]:
                return ys[j - 1] + (ys[j] - ys[j - 1]) * (target - xs[j - 1]) / (xs[j] - xs[j - 1])
        return ys[0] if xs and xs[0] >= target else None

    target = 0.9
    base = calcs_at(curves[0]["points"], target)
    savings = []
    for c in curves:
        v = calcs_at(c["points"], target)
        savings.append({"tau_over_ef": c["tau_over_ef"], "calcs_at_recall": v,
                        "fraction_of_tau0": None if (v is None or not base) else round(v / base, 4)})
    threshold = None
    for a, b in zip(savings, savings[1:]):
        fa, fb = a["fraction_of_tau0"], b["fraction_of_tau0"]
        if fa is not None and fb is not None and fa > 0.5 >= fb:
            threshold = a["tau_over_ef"] + (b["tau_over_ef"] - a["tau_over_ef"]) * (fa - 0.5) / (fa - fb)
            break
    print(json.dumps({"metric": "distance calculations vs recall by tau/ef (final stage alone)",
                      "workload": args.workload, "n": idx.n, "d": idx.d, "nq": nq, "recall_target": target,
                      "curves": curves, "savings": savings, "acceleration_threshold_2x": threshold,
                      "data": "synthetic"}), flush=True)
    return 0


def run_ablation(args):
    """Component ablation in the manner of the paper's ablation table (Sec. 6.3):
    at one ef, recall@10 and batch QPS of the full staged search, of FES seeds
    T in {1, 4, 16}, without FES (the first entry), without stage (1)
    (graceful degradation, Sec. 4.1) and without stage (2)'s expansions."""
    import torch
    from paper_2503_21206_b300 import pilot
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq)
    nq, k = len(Q), w.k
    ef = args.ef or 256
    g = pilot.load_index_data(idx)
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    cnt = torch.empty((nq, 8), dtype=torch.int32, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    kms = np.zeros(3, np.float32)
    variants = [("staged (paper)", {}), ("fes_seeds=4", {"fes_seeds": 4}), ("fes_seeds=16", {"fes_seeds": 16}),
                ("clustered FES (r = 32)", {"use_fes": 2}),
                ("no FES (first entry)", {"use_fes": 0}), ("no stage (2) expansions", {"stage2_expansions": 0}),
                ("no stage (1) (plain final stage)", {"stage1": 0, "stage2_expansions": 0})]
    rows = []
    for name, sw in variants:
        opts = pilot.pilot_search_options_default()
        for key, v in sw.items():
            setattr(opts, key, v)

        def search(counters=None):
            return pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, options=opts, counters=counters,
                                         kernel_ms=kms)

        search(cnt)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt, k)
        c = cnt.cpu().numpy().astype(np.float64)
        step_ms, search_ms = timed_steps(search, stream, flush, args.steps, args.warmup, kms)
        rows.append({"variant": name, "recall@10": round(rec, 5), "qps": nq / (step_ms / 1000.0),
                     "search_kernel_ms": search_ms,
                     "mean_counters": {n: round(float(c[:, i].mean()), 1) for i, n in
                                       enumerate(["exp1", "dist1", "exp2", "dist2", "exp3", "dist3", "rerank"])}})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"metric": "ablation at fixed ef", "workload": args.workload, "n": idx.n, "nq": nq, "k": k,
                      "ef": ef, "data": "synthetic", "rows": rows}), flush=True)
    return 0


def run_pilot(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    from paper_2503_21206_b300 import pilot
    w, idx, Q, gt = load_workload(args.workload, args.n, args.nq, verbose=(rank == 0))
    nq, k = len(Q), w.k
    g = pilot.load_index_data(idx, full_vecs_host=args.full_host)
    stream = torch.cuda.Stream(device=device)
    qd = torch.from_numpy(Q).to(device)
    ids = torch.empty((nq, k), dtype=torch.int32, device=device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=device)
    cnt = torch.empty((nq, 8), dtype=torch.int32, device=device)
    kms = np.zeros(3, np.float32)
    opts = pilot.pilot_search_options_default()
    if args.warps_per_block:
        opts.warps_per_block = args.warps_per_block
    if args.stage_rows:
        opts.stage_rows = args.stage_rows

    def search(q, ef, o_ids, o_d, counters=None, timing=kms):
        return pilot.pilot_search_ex(g, q, k, ef, o_ids, o_d, stream, options=opts, counters=counters,
                                     kernel_ms=timing)

    # operating point: the smallest swept ef reaching recall@10 >= 0.95; one
    # untimed call first, so the sweep's times exclude the workspace
    # allocation and module loading of the first call
    efs = [args.ef] if args.ef else list(w.efs) + [e for e in EXTRA_EFS if e > max(w.efs)]
    search(qd, efs[0], ids, dists, cnt)
    torch.cuda.synchronize()
    sweep, ef = [], None
    for cand in efs:
        search(qd, cand, ids, dists, cnt)
        torch.cuda.synchronize()
        rec = recall_at_k(ids.cpu().numpy(), gt, k)
        sweep.append({"ef": cand, "recall@10": round(rec, 5), "search_ms": round(float(kms[2]), 4)})
        ef = cand
        if rec >= 0.95:
            break
    # the library's autotuner picks the launch shape for this ef on the batch
    # itself (it leaves results unchanged; explicit --warps-per-block /
    # --stage-rows still override it)
    tuned = None
    if not args.no_autotune:
        tuned = pilot.pilot_autotune(g, qd, k, ef, stream, options=opts)
    search(qd, ef, ids, dists, cnt)
    torch.cuda.synchronize()
    counters = cnt.cpu().numpy()
    recall = recall_at_k(ids.cpu().numpy(), gt, k)
    alg_bytes = algorithmic_bytes(counters, k, idx)

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    for _ in range(args.warmup):
        search(qd, ef, ids, dists)

    # ---- device-timed steps: inputs resident in HBM, L2 flushed between steps
    step_ms, search_ms = [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(device)
    torch.cuda.synchronize()
    with ClockSampler(device.index or 0) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            ev0.record(stream)
            search(qd, ef, ids, dists)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            search_ms.append(float(kms[2]))
        torch.cuda.synchronize()
        barrier(device)
        t_wall = time.perf_counter() - t_wall
    clocks = clk.summary()
    max_s = reduce_max(sum(step_ms) / 1000.0, device)
    value = aggregate_throughput(nq * args.steps, ws, max_s)

    # ---- end to end through the C ABI with pinned HOST buffers (copies timed)
    qh = torch.from_numpy(Q).pin_memory()
    ids_h = torch.empty((nq, k), dtype=torch.int32).pin_memory()
    dists_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    e2e_s = []
    for _ in range(max(1, args.steps)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pilot.pilot_search(g, qh, k, ef, ids_h, dists_h, stream)
        e2e_s.append(time.perf_counter() - t0)
    e2e_value = aggregate_throughput(nq * len(e2e_s), ws, reduce_max(sum(e2e_s), device))
    e2e_recall = recall_at_k(ids_h.numpy(), gt, k)

    # ---- per-stage split: stage (1) + re-rank alone (stages (2)(3) off), the
    # rest by difference; algorithmic bytes from each run's own counters
    o1 = pilot.pilot_search_options_default()
    for key in ("warps_per_block", "stage_rows"):
        setattr(o1, key, getattr(opts, key))
    o1.stage2_expansions, o1.stage3 = 0, 0
    cnt1 = torch.empty_like(cnt)
    pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, options=o1, counters=cnt1, kernel_ms=kms)
    torch.cuda.synchronize()
    c1 = cnt1.cpu().numpy()
    _, s1_ms = timed_steps(lambda: pilot.pilot_search_ex(g, qd, k, ef, ids, dists, stream, options=o1,
                                                         kernel_ms=kms), stream, flush, args.steps, 3, kms)
    s1_bytes = algorithmic_bytes(c1, k, idx)
    stage_split = {"stage1_rerank_ms": s1_ms, "stage1_rerank_gbs": s1_bytes / (s1_ms / 1000.0) / 1e9,
                   "stage23_ms_by_difference": None, "stage23_gbs_by_difference": None}
    serving = None
    if not args.no_serving:
        serving = serving_run(pilot, g, Q, gt, args.serve_rate, args.serve_requests, max_ef=512, max_k=100,
                              expansions_per_step=args.serve_budget)
        # capacity: the operating point's k and ef offered at twice the batch rate
        cap_rate = 2.0 * aggregate_throughput(nq * args.steps, 1, sum(step_ms) / 1000.0)
        serving["capacity"] = serving_run(pilot, g, Q, gt, cap_rate, min(int(cap_rate * 0.5), 150_000),
                                          fixed_ef=ef, max_ef=512, max_k=100,
                                          expansions_per_step=args.serve_budget)
    forms = None
    if not args.no_forms and ws == 1:
        forms = forms_summary(args)
    peak, peak_kind = measured_peaks()
    mean_search_ms = statistics.mean(search_ms)
    achieved = alg_bytes / (mean_search_ms / 1000.0) / 1e9
    if mean_search_ms > s1_ms:
        stage_split["stage23_ms_by_difference"] = mean_search_ms - s1_ms
        stage_split["stage23_gbs_by_difference"] = (alg_bytes - s1_bytes) / ((mean_search_ms - s1_ms) / 1000.0) / 1e9
    stage_split["stage1_rerank_frac"] = stage_split["stage1_rerank_gbs"] / peak
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(idx, Q, k, ef)
    c = counters.astype(np.float64)
    line = {
        "metric": "QPS@recall10=0.95", "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * max_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": idx.n, "d": idx.d, "dp": idx.dp, "nq": nq, "k": k, "ef": ef,
                   "recall@10": round(recall, 5), "R": int(idx.graph.shape[1]), "sample_ratio": w.sample_ratio,
                   "n_entry": int(len(idx.entry_ids)), "reduced_dtype": idx.reduced_dtype,
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)", "sweep": sweep,
                   "parallelism": f"replicas x{ws}", "autotuned": tuned,
                   "full_vecs": "pinned host memory" if args.full_host else "device",
                   "mean_counters": {name: round(float(c[:, i].mean()), 2) for i, name in
                                     enumerate(["exp1", "dist1", "exp2", "dist2", "exp3", "dist3", "rerank"])}},
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": int(nq * idx.d * 4),
                "d2h_bytes_per_step": int(nq * k * 8), "recall@10": round(e2e_recall, 5)},
        "gpu_launches": 3 * args.steps,
        "roofline": {"kernel": "search_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": profiled_traffic(args.workload, ef, nq),
                     "peak_source": f"{peak_kind} hbm_gbs (copy)", "algorithmic_bytes_per_launch": alg_bytes,
                     "mean_kernel_ms": mean_search_ms},
        "kernel_ms": {"project": float(kms[0]), "fes_scores": float(kms[1]), "search": mean_search_ms},
        "stage_split": stage_split,
        "clocks": clocks, "wall_s_timed": round(t_wall, 4),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if serving is not None:
        line["serving"] = serving
    if forms is not None:
        line["forms"] = forms
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description="PilotANN staged search benchmark")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pilot", "reference"], default="pilot")
    ap.add_argument("--workload", default="c2_aniso_1m_d96")
    ap.add_argument("--ef", type=int, default=0, help="a fixed ef instead of the recall-0.95 sweep")
    ap.add_argument("--n", type=int, default=None, help="smaller base set (profiling cases)")
    ap.add_argument("--nq", type=int, default=None, help="queries: fewer takes a prefix, more draws them from the same generator (profiling cases)")
    ap.add_argument("--warps-per-block", type=int, default=0)
    ap.add_argument("--stage-rows", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (continuous batching) run")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the compact served BF16 vs FP32 comparison on the 768-d workload's prefix")
    ap.add_argument("--serve-rate", type=float, default=50_000.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-requests", type=int, default=100_000)
    ap.add_argument("--serve-budget", type=int, default=4096, help="expansions per request per step")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--full-host", action="store_true",
                    help="memory-bounded form: full vectors in pinned host memory, read over the host link")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="serving at each of --serve-rates (mixed k and ef) beside the batch operating points")
    ap.add_argument("--serve-rates", default="20000,50000,100000,200000")
    ap.add_argument("--sweep-sub", action="store_true",
                    help="sampling ratio x SVD ratio sweep of the staged search (QPS at recall 0.95)")
    ap.add_argument("--sample-ratios", default="0.25,0.5,1.0")
    ap.add_argument("--svd-ratios", default="0.25,0.5,1.0")
    ap.add_argument("--tau", action="store_true",
                    help="the tau/ef analysis: final stage seeded with tau true neighbours + random nodes")
    ap.add_argument("--ablation", action="store_true",
                    help="component ablation (FES seeds, stages on/off) at --ef (default 256)")
    ap.add_argument("--memory-bounded", action="store_true",
                    help="the memory-bounded configuration (full vectors in pinned host memory): QPS at recall "
                         "0.9 / 0.95 and a mixed-ef serving run; e.g. --workload c5_powerlaw_25m_d768 --nq 2000")
    ap.add_argument("--gather-ceiling", action="store_true",
                    help="random-row read bandwidth for the row sizes the search reads (context for the roofline)")
    ap.add_argument("--forms", action="store_true",
                    help="compare the reduced-row precision forms and the plain form (one GPU)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.serve_sweep:
        return run_serve_sweep(args)
    if args.memory_bounded:
        return run_memory_bounded(args)
    if args.gather_ceiling:
        return run_gather_ceiling(args)
    if args.tau:
        return run_tau(args)
    if args.sweep_sub:
        return run_sweep_sub(args)
    return run_forms(args) if args.forms else run_pilot(args)


if __name__ == "__main__":
    sys.exit(main())
