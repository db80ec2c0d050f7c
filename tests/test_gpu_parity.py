"""GPU path vs the oracle, element by element, through the C ABI.

Both sides round each distance once to FP32, break ties by id and keep exact
visited sets, so ids, distances and per-stage counters must be identical.  The tolerance the paper's
reading allows (ties within 1e-5 relative) is kept as the fallback check
``assert_parity`` reports against when anything differs."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2503_21206_b300 import index_build, synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def pilot(torch_cuda):
    from paper_2503_21206_b300 import build
    build.build()
    from paper_2503_21206_b300 import pilot as p
    return p


def oracle_index(idx):
    dt = {"f32": oracle.DTYPE_F32, "bf16": oracle.DTYPE_BF16, "fp8": oracle.DTYPE_FP8}[idx.reduced_dtype]
    return oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, dt,
                              idx.reduced_scales, idx.full, idx.entry_ids, idx.metric, idx.entry_cluster,
                              idx.cluster_centroids)


def gpu_search(pilot, torch, gidx, Q, k, ef, device=True, **opts):
    o = pilot.pilot_search_options_default()
    for key, v in opts.items():
        setattr(o, key, int(v))
    nq = len(Q)
    if device:
        q = torch.from_numpy(Q).cuda()
        ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
        dists = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        cnt = torch.empty((nq, 8), dtype=torch.int32, device="cuda")
        pilot.pilot_search_ex(gidx, q, k, ef, ids, dists, options=o, counters=cnt)
        torch.cuda.synchronize()
        return ids.cpu().numpy(), dists.cpu().numpy(), cnt.cpu().numpy()
    cnt = np.empty((nq, 8), np.int32)
    ids, dists = pilot.pilot_search_ex(gidx, np.ascontiguousarray(Q), k, ef, options=o, counters=cnt)
    return ids, dists, cnt


def assert_parity(ids, dists, ref_ids, ref_dists, rel_tie=1e-5):
    """ids equal except where the two distances tie within rel_tie."""
    bad = []
    for i in range(ids.shape[0]):
        if np.array_equal(ids[i], ref_ids[i]) and np.array_equal(dists[i], ref_dists[i]):
            continue
        for j in range(ids.shape[1]):
            if ids[i, j] == ref_ids[i, j]:
                continue
            a, b = float(dists[i, j]), float(ref_dists[i, j])
            if not (np.isfinite(a) and np.isfinite(b) and abs(a - b) <= rel_tie * max(abs(a), abs(b))):
                bad.append((i, j, int(ids[i, j]), int(ref_ids[i, j]), a, b))
    assert not bad, f"{len(bad)} mismatches, first: {bad[:5]}"


@pytest.fixture(scope="module")
def c1(pilot):
    w = synth.WORKLOADS["c1_mixture_20k_d96"]
    idx, Q, red32, V = index_build.build_workload(w)
    return w, idx, Q, red32, pilot.load_index_data(idx)


def test_c1_full_parity(c1, pilot, torch_cuda):
    """The tiny parity workload at its stated size (N=20k, 200 queries, k=10,
    ef=64): ids, distances and per-stage counters identical."""
    w, idx, Q, _, g = c1
    ref = oracle.search(oracle_index(idx), Q, w.k, 64)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, w.k, 64)
    assert_parity(ids, dists, ref["ids"], ref["dists"])
    assert np.array_equal(ids, ref["ids"])
    assert np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


@pytest.mark.parametrize("k, ef", [(1, 1), (1, 32), (10, 10), (10, 33), (32, 128), (100, 512)])
def test_c1_k_ef_grid(c1, pilot, torch_cuda, k, ef):
    w, idx, Q, _, g = c1
    Qs = Q[:37]
    ref = oracle.search(oracle_index(idx), Qs, k, ef)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Qs, k, ef)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


@pytest.mark.parametrize("opts", [dict(stage1=0), dict(stage2_expansions=0), dict(stage3=0), dict(use_fes=0),
                                  dict(stage1=0, stage2_expansions=0), dict(stage2_expansions=5)])
def test_stage_switches(c1, pilot, torch_cuda, opts):
    w, idx, Q, _, g = c1
    Qs = Q[:40]
    oopts = dict(stage1=bool(opts.get("stage1", 1)), stage2_expansions=opts.get("stage2_expansions", 2),
                 stage3=bool(opts.get("stage3", 1)), use_fes=bool(opts.get("use_fes", 1)))
    ref = oracle.search(oracle_index(idx), Qs, 10, 64, **oopts)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Qs, 10, 64, **opts)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


def test_visited_epochs_wrap(c1, pilot, torch_cuda):
    """Visited sets carry an epoch tag, and a slot's table is cleared when its
    epochs run out.  With the cycle shortened to 3 sets
    (PILOT_VISITED_EPOCH_CYCLE, read at load), 40 back-to-back searches (two
    sets per query) wrap every used slot many times; every repetition must
    return the oracle's results."""
    w, idx, Q, _, _ = c1
    os.environ["PILOT_VISITED_EPOCH_CYCLE"] = "3"
    try:
        g = pilot.load_index_data(idx)
    finally:
        del os.environ["PILOT_VISITED_EPOCH_CYCLE"]
    ref = oracle.search(oracle_index(idx), Q[:24], 10, 64)
    for rep in range(40):
        ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q[:24], 10, 64)
        assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"]), rep
        assert np.array_equal(cnt, ref["counters"]), rep
    g.free()


def test_visited_table_overflow_keeps_results(c1, pilot, torch_cuda):
    """The exact-visited reading of Sec. 4.3: a visited insertion that finds no
    room is treated as "not visited".  A 256-entry table cannot hold the
    thousand-odd nodes a stage visits at ef = 128, so many insertions fail;
    such a node is scored again when met again and the merge drops its equal
    key, so ids, distances and expansion counts stay the oracle's, the
    distance counts can only grow, and status word 7 counts the failures."""
    w, idx, Q, _, g = c1
    Qs = Q[:48]
    ref = oracle.search(oracle_index(idx), Qs, 10, 128)
    o = pilot.pilot_search_options_default()
    o.visited_entries = 256
    status = np.zeros(8, np.int32)
    o.status_words = status.ctypes.data
    cnt = np.empty((len(Qs), 8), np.int32)
    ids, dists = pilot.pilot_search_ex(g, np.ascontiguousarray(Qs), 10, 128, options=o, counters=cnt)
    assert status[7] > 0
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    rc = ref["counters"]
    for c in (0, 2, 4, 6, 7):   # expansions, re-ranked count, entry
        assert np.array_equal(cnt[:, c], rc[:, c]), c
    for c in (1, 3, 5):         # distances
        assert np.all(cnt[:, c] >= rc[:, c]), c
    assert (cnt[:, [1, 3, 5]] > rc[:, [1, 3, 5]]).any()
    # the automatic size holds every stage: counters equal, no failure
    o.visited_entries = 0
    status[:] = 0
    ids, dists = pilot.pilot_search_ex(g, np.ascontiguousarray(Qs), 10, 128, options=o, counters=cnt)
    assert status[7] == 0 and np.array_equal(cnt, rc) and np.array_equal(ids, ref["ids"])
    with pytest.raises(pilot.PilotError) as e:
        o.visited_entries = 300
        pilot.pilot_search_ex(g, np.ascontiguousarray(Qs), 10, 128, options=o)
    assert e.value.status == pilot.PILOT_EINVAL


def test_host_and_device_buffers_agree(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    a = gpu_search(pilot, torch_cuda, g, Q[:64], 10, 64, device=True)
    b = gpu_search(pilot, torch_cuda, g, Q[:64], 10, 64, device=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_ragged_and_empty_batches(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    for nq in (0, 1, 31, 33, 129):
        Qs = np.ascontiguousarray(Q[:nq])
        ids, dists, _ = gpu_search(pilot, torch_cuda, g, Qs, 10, 64, device=False)
        if nq:
            ref = oracle.search(oracle_index(idx), Qs, 10, 64)
            assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])


def test_nonfinite_query_rejected_others_answered(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    Qs = Q[:8].copy()
    Qs[3, 5] = np.nan
    with pytest.raises(pilot.PilotError) as e:
        pilot.pilot_search(g, Qs, 10, 64)
    assert e.value.status == pilot.PILOT_EINVAL
    ids = np.empty((8, 10), np.int32)
    dists = np.empty((8, 10), np.float32)
    with pytest.raises(pilot.PilotError):
        pilot.pilot_search(g, Qs, 10, 64, ids, dists)
    ref = oracle.search(oracle_index(idx), np.delete(Qs, 3, 0), 10, 64)
    assert np.array_equal(np.delete(ids, 3, 0), ref["ids"])
    assert np.all(ids[3] == -1) and np.all(np.isinf(dists[3]))


def test_argument_validation(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    for k, ef in ((0, 10), (11, 10), (10, 513)):
        with pytest.raises(pilot.PilotError) as e:
            pilot.pilot_search(g, Q[:2], k, ef)
        assert e.value.status == pilot.PILOT_EINVAL


@pytest.mark.parametrize("name", ["alg1_path_line.json", "alg1_local_minimum.json", "alg1_two_cliques.json"])
def test_golden_traces_on_gpu(pilot, torch_cuda, name):
    gdata = json.load(open(os.path.join(GOLDEN, name)))
    X = np.asarray(gdata["points"], np.float32)
    n, d = X.shape
    G = np.asarray(gdata["graph"], np.int32)
    g = pilot.pilot_index_load(G, np.ones(n, np.uint8), G, np.eye(d), X, X, np.asarray([gdata["entry"]], np.int32))
    for case in gdata["cases"]:
        ids, dists, cnt = gpu_search(pilot, torch_cuda, g, np.asarray([gdata["query"]], np.float32), case["k"],
                                     case["ef"], stage1=0, stage2_expansions=0, use_fes=0)
        assert ids[0].tolist() == case["ids"]
        np.testing.assert_array_equal(dists[0], np.asarray(case["dists"], np.float32))
        assert cnt[0, 4] == case["expansions"] and cnt[0, 5] == case["distances"]


def test_seeded_golden_on_gpu(pilot, torch_cuda):
    """The hand trace of the seeded final stage (tests/golden/seeded_path_line.json)."""
    line = json.load(open(os.path.join(GOLDEN, "alg1_path_line.json")))
    gd = json.load(open(os.path.join(GOLDEN, "seeded_path_line.json")))
    X = np.asarray(line["points"], np.float32)
    n, d = X.shape
    G = np.asarray(line["graph"], np.int32)
    g = pilot.pilot_index_load(G, np.ones(n, np.uint8), G, np.eye(d), X, X, np.asarray([line["entry"]], np.int32))
    seeds = np.asarray([gd["seeds"]], np.int32)
    o = pilot.pilot_search_options_default()
    o.stage1, o.stage2_expansions = 0, 0
    o.seed_ids, o.seed_count = seeds.ctypes.data, seeds.shape[1]
    cnt = np.empty((1, 8), np.int32)
    ids, dists = pilot.pilot_search_ex(g, np.asarray([line["query"]], np.float32), gd["k"], gd["ef"], options=o,
                                       counters=cnt)
    assert ids[0].tolist() == gd["ids"]
    np.testing.assert_array_equal(dists[0], np.asarray(gd["dists"], np.float32))
    assert cnt[0].tolist() == gd["counters"]


def test_golden_staged_on_gpu(pilot, torch_cuda):
    gd = json.load(open(os.path.join(GOLDEN, "staged_2d.json")))
    X = np.asarray(gd["points"], np.float32)
    mask = np.asarray(gd["mask"], np.uint8)
    basis = np.asarray(gd["basis"], np.float64)
    red = (X[mask == 1].astype(np.float64) @ basis).astype(np.float32)
    g = pilot.pilot_index_load(np.asarray(gd["graph"], np.int32), mask, np.asarray(gd["subgraph"], np.int32), basis,
                               red, X, np.asarray(gd["entries"], np.int32))
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, np.asarray([gd["query"]], np.float32), gd["k"], gd["ef"])
    assert ids[0].tolist() == gd["ids"]
    np.testing.assert_array_equal(dists[0], np.asarray(gd["dists"], np.float32))
    assert cnt[0].tolist() == gd["counters"]


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_low_precision_reduced_rows(c1, pilot, torch_cuda, dtype):
    """BF16 / FP8-E4M3 reduced rows: both sides decode the same codes exactly
    and accumulate exactly, so results stay identical."""
    w, idx, Q, red32, _ = c1
    lp = idx.with_reduced(dtype, red32)
    g = pilot.load_index_data(lp)
    ref = oracle.search(oracle_index(lp), Q[:100], 10, 64)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q[:100], 10, 64)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_inner_product_metric(pilot, torch_cuda, dtype):
    w = synth.WORKLOADS["c3_powerlaw_2m_d768"]
    idx, Q, red32, _ = index_build.build_workload(w, n=6000, nq=40, reduced_dtype=dtype)
    g = pilot.load_index_data(idx)
    ref = oracle.search(oracle_index(idx), Q, 10, 64)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 64)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


@pytest.mark.parametrize("stage_rows", [4, 8, 12, 20])
def test_wide_rows_multi_pass(pilot, torch_cuda, stage_rows):
    """d = 768: a batch of up to 32 full rows (3 KB each) is gathered in
    several passes through two half-buffers; every staging size gives the
    oracle's results."""
    w = synth.WORKLOADS["c3_powerlaw_2m_d768"]
    idx, Q, red32, _ = index_build.build_workload(w, n=4000, nq=24, reduced_dtype="bf16")
    g = pilot.load_index_data(idx)
    ref = oracle.search(oracle_index(idx), Q, 10, 48)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 48, stage_rows=stage_rows)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


@pytest.mark.parametrize("T", [2, 5, 16])
def test_fes_seeds_parity(c1, pilot, torch_cuda, T):
    """Top-T FES seeding: the GPU seeds stage (1) with the same T entries and
    then follows the same path."""
    w, idx, Q, _, g = c1
    ref = oracle.search(oracle_index(idx), Q, 10, 64, fes_seeds=T)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 64, fes_seeds=T)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


def test_fes_seeds_without_fes_and_inner_product(pilot, torch_cuda):
    w = synth.WORKLOADS["c3_powerlaw_2m_d768"]
    idx, Q, _, _ = index_build.build_workload(w, n=5000, nq=24, reduced_dtype="bf16")
    g = pilot.load_index_data(idx)
    for use_fes, T in ((True, 4), (False, 3)):
        ref = oracle.search(oracle_index(idx), Q, 10, 48, use_fes=use_fes, fes_seeds=T)
        ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 48, use_fes=use_fes, fes_seeds=T)
        assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
        assert np.array_equal(cnt, ref["counters"])


def test_fes_seed_ties_take_the_exact_scan(pilot, torch_cuda):
    """Entries with identical vectors tie on distance: the 16 scored survivors
    cannot certify the T best, so the warp scans the entry set exactly and
    breaks the ties by id, like the oracle."""
    rng = np.random.default_rng(11)
    base = rng.standard_normal((12, 96)).astype(np.float32)
    X = np.repeat(base, 200, axis=0)           # 2400 rows, each vector 200 times (~50 entries each)
    Q = (base + 0.05 * rng.standard_normal((12, 96))).astype(np.float32)
    idx = index_build.build_index(X, 16, 16, 0.5, 32, 600, 0, 5, 6, "f32")
    g = pilot.load_index_data(idx)
    for T in (1, 8):
        ref = oracle.search(oracle_index(idx), Q, 10, 32, fes_seeds=T)
        o = pilot.pilot_search_options_default()
        o.fes_seeds = T
        status = np.zeros(8, np.int32)
        o.status_words = status.ctypes.data
        cnt = np.empty((len(Q), 8), np.int32)
        ids, dists = pilot.pilot_search_ex(g, Q, 10, 32, options=o, counters=cnt)
        assert status[3] > 0, "no query took the exact entry scan"
        assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
        assert np.array_equal(cnt, ref["counters"])


def test_fes_seeds_out_of_range(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    for bad in (-1, 17):
        with pytest.raises(pilot.PilotError):
            gpu_search(pilot, torch_cuda, g, Q[:4], 10, 64, fes_seeds=bad)


def _tau_seeds(gt, n, ef, tau, seed):
    """tau true neighbours plus ef - tau distinct random other nodes per row."""
    rng = np.random.default_rng(seed)
    rows = []
    for t in gt:
        known = t[:tau].tolist()
        pool = rng.permutation(n)
        rest = [int(v) for v in pool[: ef + tau] if int(v) not in set(known)][: ef - tau]
        rows.append(known + rest)
    return np.asarray(rows, np.int32)


@pytest.mark.parametrize("tau", [0, 8, 16])
def test_seeded_final_stage_parity(c1, pilot, torch_cuda, tau):
    """Sec. 4.2's experiment through the C ABI: the final stage alone from tau
    known neighbours plus random nodes equals the oracle's run."""
    w, idx, Q, _, g = c1
    ef = 64
    gt, _ = oracle.bruteforce(idx.full, Q, ef)
    seeds = _tau_seeds(gt, idx.n, ef, tau, 3)
    seeds[::7, -1] = -1                                   # skipped entries
    ref = oracle.search(oracle_index(idx), Q, 10, ef, seed_ids=seeds)
    o = pilot.pilot_search_options_default()
    o.stage1, o.stage2_expansions = 0, 0
    o.seed_ids, o.seed_count = seeds.ctypes.data, seeds.shape[1]
    cnt = np.empty((len(Q), 8), np.int32)
    ids, dists = pilot.pilot_search_ex(g, Q, 10, ef, options=o, counters=cnt)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


def test_seed_ids_validation(c1, pilot, torch_cuda):
    w, idx, Q, _, g = c1
    good = np.tile(np.arange(8, dtype=np.int32), (4, 1))

    def run(seeds, **kw):
        o = pilot.pilot_search_options_default()
        o.stage1, o.stage2_expansions = 0, 0
        for key, v in kw.items():
            setattr(o, key, v)
        o.seed_ids, o.seed_count = seeds.ctypes.data, seeds.shape[1]
        return pilot.pilot_search_ex(g, Q[:4], 10, 16, options=o)

    run(good)
    for bad in (dict(stage1=1), dict(stage3=0), dict(stage2_expansions=2)):
        with pytest.raises(pilot.PilotError):
            run(good, **bad)
    rep = good.copy()
    rep[1, 3] = rep[1, 2]
    out = good.copy()
    out[2, 0] = idx.n
    wide = np.tile(np.arange(17, dtype=np.int32), (4, 1))
    for seeds in (rep, out, wide):
        with pytest.raises(pilot.PilotError):
            run(seeds)


def test_full_vectors_in_host_memory(c1, pilot, torch_cuda, tmp_path):
    """The memory-bounded form: full vectors in pinned host memory, read by the
    re-rank and stages (2)(3) over the host link.  Results equal the oracle's
    (and the device-resident index's), through both loaders, and through the
    server."""
    w, idx, Q, _, g_dev = c1
    g = pilot.load_index_data(idx, full_vecs_host=True)
    ref = oracle.search(oracle_index(idx), Q, 10, 64)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 64)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])
    assert g.info()["device_bytes"] < g_dev.info()["device_bytes"]
    index_build.save_index(idx, str(tmp_path))
    g2 = pilot.pilot_index_load_files(str(tmp_path), pilot.LOAD_FULL_VECS_HOST)
    ids2, dists2, _ = gpu_search(pilot, torch_cuda, g2, Q[:40], 10, 64)
    assert np.array_equal(ids2, ref["ids"][:40]) and np.array_equal(dists2, ref["dists"][:40])
    srv = pilot.pilot_serve_create(g, max_ef=64, max_k=10, expansions_per_step=16)
    try:
        tickets = [srv.submit(Q[i], 10, 64) for i in range(24)]
        for i, t in enumerate(tickets):
            sid, sd = srv.wait(t, 10)
            assert np.array_equal(sid, ref["ids"][i]) and np.array_equal(sd, ref["dists"][i])
    finally:
        srv.destroy()
    with pytest.raises(pilot.PilotError):
        pilot.pilot_index_load_files(str(tmp_path), 2)


@pytest.mark.parametrize("T", [1, 4])
def test_clustered_fes_parity(c1, pilot, torch_cuda, T):
    """Clustered FES (Sec. 5, r = 32 coarse clusters): the GPU routes each
    query to the same cluster and seeds stage (1) like the oracle."""
    w, idx, Q, _, g = c1
    assert idx.cluster_centroids is not None and idx.cluster_centroids.shape[0] == 32
    ref = oracle.search(oracle_index(idx), Q, 10, 64, use_fes=2, fes_seeds=T)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 64, use_fes=2, fes_seeds=T)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])


def test_clustered_fes_inner_product_files_and_errors(pilot, torch_cuda, tmp_path):
    w = synth.WORKLOADS["c3_powerlaw_2m_d768"]
    idx, Q, _, _ = index_build.build_workload(w, n=5000, nq=24, reduced_dtype="bf16")
    index_build.save_index(idx, str(tmp_path))
    g = pilot.pilot_index_load_files(str(tmp_path))
    ref = oracle.search(oracle_index(idx), Q, 10, 48, use_fes=2, fes_seeds=2)
    ids, dists, cnt = gpu_search(pilot, torch_cuda, g, Q, 10, 48, use_fes=2, fes_seeds=2)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"])
    assert np.array_equal(cnt, ref["counters"])
    bare = pilot.pilot_index_load(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, idx.full,
                                  idx.entry_ids, metric=idx.metric, reduced_dtype=idx.reduced_dtype)
    with pytest.raises(pilot.PilotError):
        gpu_search(pilot, torch_cuda, bare, Q[:4], 10, 48, use_fes=2)
    bad = idx.entry_cluster.copy()
    bad[bad == 3] = 4                                   # cluster 3 left empty
    with pytest.raises(pilot.PilotError):
        pilot.pilot_index_load(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, idx.full,
                               idx.entry_ids, metric=idx.metric, reduced_dtype=idx.reduced_dtype,
                               entry_cluster=bad, cluster_centroids=idx.cluster_centroids)


def test_load_from_files(c1, pilot, torch_cuda, tmp_path):
    w, idx, Q, _, g = c1
    index_build.save_index(idx, str(tmp_path))
    g2 = pilot.pilot_index_load_files(str(tmp_path))
    a = gpu_search(pilot, torch_cuda, g, Q[:20], 10, 64)
    b = gpu_search(pilot, torch_cuda, g2, Q[:20], 10, 64)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_short_results_are_padded(pilot, torch_cuda):
    """Fewer than k reachable nodes: -1 ids and +inf distances."""
    X = np.arange(5, dtype=np.float32)[:, None] * np.ones((1, 4), np.float32)
    G = np.full((5, 2), -1, np.int32)
    G[0, 0], G[1, 0] = 1, 2   # 0 -> 1 -> 2; 3 and 4 unreachable
    g = pilot.pilot_index_load(G, np.ones(5, np.uint8), G, np.eye(4), X, X, np.asarray([0], np.int32))
    ids, dists, _ = gpu_search(pilot, torch_cuda, g, np.zeros((1, 4), np.float32), 5, 8)
    assert ids[0].tolist() == [0, 1, 2, -1, -1]
    assert np.all(np.isinf(dists[0, 3:]))


def test_large_id_space_uses_the_widest_visited_quotients(pilot, torch_cuda):
    """Visited entries store a node's quotient within its bucket (at most 13
    bits) rather than its id, so an index whose ids need 23 bits gets tables
    of at least 2^14 words (1,024 buckets).  On a 4.2M-node index (a ring of
    16 seeded random offsets, random 32-d rows, every node sampled), a search
    whose table is capped at that floor uses 13-bit quotients, the widest the
    encoding allows, and must still return the oracle's ids, distances and
    counters with no insertion left without room; a cap below the floor is
    rejected."""
    rng = np.random.default_rng(23)
    n, d, R = (1 << 22) + 4096, 32, 16
    offsets = rng.choice(np.arange(1, n, dtype=np.int64), size=R, replace=False)
    graph = ((np.arange(n, dtype=np.int64)[:, None] + offsets[None, :]) % n).astype(np.int32)
    full = rng.standard_normal((n, d), dtype=np.float32)
    mask = np.ones(n, np.uint8)
    basis = np.eye(d, dtype=np.float64)
    entries = np.arange(256, dtype=np.int32)
    Q = rng.standard_normal((8, d), dtype=np.float32)
    g = pilot.pilot_index_load(graph, mask, graph, basis, full, full, entries)
    oi = oracle.OracleIndex(graph, mask, graph, basis, full, oracle.DTYPE_F32, None, full, entries, 0)
    ref = oracle.search(oi, Q, 10, 64)
    floor_words = 1 << (23 - 9)
    for cap in (0, floor_words):
        o = pilot.pilot_search_options_default()
        o.visited_entries = cap
        status = np.zeros(8, np.int32)
        o.status_words = status.ctypes.data
        cnt = np.empty((len(Q), 8), np.int32)
        ids, dists = pilot.pilot_search_ex(g, Q, 10, 64, options=o, counters=cnt)
        assert np.array_equal(ids, ref["ids"]) and np.array_equal(dists, ref["dists"]), cap
        assert np.array_equal(cnt, ref["counters"]), cap
        assert status[7] == 0, cap
    with pytest.raises(pilot.PilotError) as e:
        o = pilot.pilot_search_options_default()
        o.visited_entries = floor_words // 2
        pilot.pilot_search_ex(g, Q, 10, 64, options=o)
    assert e.value.status == pilot.PILOT_EINVAL
    g.free()
