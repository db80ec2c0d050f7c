"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
traces of Algorithm 1 and of the staged search (tests/golden/), closed forms of
the SVD projection (Sec. 4.1 (1)), the brute-force limit of the search, the
dense-FES special case (Table 2, "FES (1 block)") and library routines
(numpy FP64 arithmetic, torch number-format conversions)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2503_21206_b300 import index_build

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _plain_index(points, graph, entry, metric=0):
    """An index whose subgraph is the full graph and whose basis is I (d'=d)."""
    X = np.asarray(points, np.float32)
    n, d = X.shape
    G = np.asarray(graph, np.int32)
    return oracle.OracleIndex(G, np.ones(n, np.uint8), G, np.eye(d), X.copy(), oracle.DTYPE_F32, None, X,
                              np.asarray([entry], np.int32), metric)


@pytest.mark.parametrize("name", ["alg1_path_line.json", "alg1_local_minimum.json", "alg1_two_cliques.json"])
def test_algorithm1_hand_traces(name):
    g = json.load(open(os.path.join(GOLDEN, name)))
    ix = _plain_index(g["points"], g["graph"], g["entry"])
    for case in g["cases"]:
        r = oracle.search(ix, np.asarray([g["query"]], np.float32), case["k"], case["ef"], stage1=False,
                          stage2_expansions=0, stage3=True, use_fes=False)
        assert r["ids"][0].tolist() == case["ids"]
        np.testing.assert_allclose(r["dists"][0], case["dists"], rtol=0)
        assert r["counters"][0, 4] == case["expansions"]
        assert r["counters"][0, 5] == case["distances"]


def test_staged_search_hand_trace():
    g = json.load(open(os.path.join(GOLDEN, "staged_2d.json")))
    X = np.asarray(g["points"], np.float32)
    mask = np.asarray(g["mask"], np.uint8)
    basis = np.asarray(g["basis"], np.float64)
    red = (X[mask == 1].astype(np.float64) @ basis).astype(np.float32)
    ix = oracle.OracleIndex(np.asarray(g["graph"], np.int32), mask, np.asarray(g["subgraph"], np.int32), basis,
                            red, oracle.DTYPE_F32, None, X, np.asarray(g["entries"], np.int32), 0)
    r = oracle.search(ix, np.asarray([g["query"]], np.float32), g["k"], g["ef"], pools=True)
    assert r["pool1_ids"][0].tolist() == g["pool1"]
    np.testing.assert_allclose(r["pool1_dists"][0], g["pool1_dists"], rtol=0)
    assert r["pool2_ids"][0].tolist() == g["pool2"]
    np.testing.assert_allclose(r["pool2_dists"][0], g["pool2_dists"], rtol=0)
    assert r["ids"][0].tolist() == g["ids"]
    np.testing.assert_allclose(r["dists"][0], g["dists"], rtol=0)
    assert r["counters"][0].tolist() == g["counters"]


def test_svd_basis_orthonormal_and_distance_preserving(c1_small):
    idx, Q, red32, V = c1_small
    d = V.shape[0]
    assert np.abs(V.T @ V - np.eye(d)).max() < 1e-10
    # d' = d: projected distances equal full distances (V^T V = I, Sec. 4.1 (1))
    full = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, V, np.zeros((1, d), np.float32),
                              oracle.DTYPE_F32, None, idx.full, idx.entry_ids, 0)
    qp, _ = oracle.project(full, Q[:16])
    xp, _ = oracle.project(full, idx.full[:64])
    for i in range(16):
        proj = ((qp[i] - xp) ** 2).sum(1)
        ref = ((Q[i].astype(np.float64) - idx.full[:64].astype(np.float64)) ** 2).sum(1)
        np.testing.assert_allclose(proj, ref, rtol=1e-12)
    # d' < d: projected distance never exceeds the full distance (Pythagoras)
    qp32, _ = oracle.project(oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis,
                                                idx.reduced, 0, None, idx.full, idx.entry_ids, 0), Q[:16])
    xs = idx.full[:200].astype(np.float64)
    xsp = xs @ idx.basis
    for i in range(16):
        proj = ((qp32[i] - xsp) ** 2).sum(1)
        ref = ((Q[i].astype(np.float64) - xs) ** 2).sum(1)
        assert np.all(proj <= ref * (1 + 1e-12))


def test_projection_rounds_each_component_once(c1_small):
    idx, Q, _, _ = c1_small
    ix = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                            idx.full, idx.entry_ids, 0)
    f64, f32 = oracle.project(ix, Q)
    ref = Q.astype(np.float64) @ idx.basis
    np.testing.assert_allclose(f64, ref, rtol=0, atol=1e-12)
    assert np.array_equal(f32, ref.astype(np.float32)) or np.mean(f32 != ref.astype(np.float32)) < 1e-3


def _exact_limit_index(n, d, R, seed, metric=0, unit=False):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    if unit:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    entry = np.asarray([0], np.int32)
    G = index_build.build_graph(X, R, entry)
    V = index_build.svd_basis(X, seed)
    red = index_build.project_rows(X, V)
    ix = oracle.OracleIndex(G, np.ones(n, np.uint8), G, V, red, 0, None, X, np.arange(0, n, 7, dtype=np.int32),
                            metric)
    return ix, X, rng


@pytest.mark.parametrize("metric", [0, 1])
def test_bruteforce_limit(metric):
    """Subgraph = full graph, d' = d, ef >= N: the staged search returns the
    exact top-k (every node is reachable, so stage (1) collects all of them
    and the re-rank orders them by full distance)."""
    n, d, k = 300, 16, 10
    ix, X, rng = _exact_limit_index(n, d, 8, 11, metric=metric, unit=(metric == 1))
    Q = rng.standard_normal((20, d)).astype(np.float32)
    r = oracle.search(ix, Q, k, n)
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    for i in range(len(Q)):
        dd = ((Q64[i] - X64) ** 2).sum(1) if metric == 0 else -(X64 @ Q64[i])
        d32 = dd.astype(np.float32)
        order = np.lexsort((np.arange(n), d32))[:k]
        assert r["ids"][i].tolist() == order.tolist()
        np.testing.assert_array_equal(r["dists"][i], d32[order])
    # and against the FP64 brute force routine
    gt, _ = oracle.bruteforce(X, Q, k, metric=metric)
    assert oracle.recall_at_k(r["ids"], gt, k) == 1.0


def test_ip_and_l2_rank_alike_on_unit_vectors():
    """On unit-norm data ||q-x||^2 = 2 - 2<q,x> (|q| = 1), so L2 and IP order
    nodes identically up to rounding ties."""
    n, d, k = 300, 16, 10
    ix, X, rng = _exact_limit_index(n, d, 8, 5, metric=1, unit=True)
    Q = rng.standard_normal((20, d)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    r_ip = oracle.search(ix, Q, k, n)
    ix.metric = 0
    r_l2 = oracle.search(ix, Q, k, n)
    assert (r_ip["ids"] == r_l2["ids"]).mean() > 0.99


def test_algorithm1_reaches_everything_with_large_ef():
    """Brute force on tiny random graphs: with ef >= N, Algorithm 1 expands
    every node reachable from the entry, so its result is the exact top-k
    among the reachable nodes."""
    rng = np.random.default_rng(3)
    for trial in range(30):
        n, d, R = int(rng.integers(2, 40)), int(rng.integers(1, 5)), int(rng.integers(1, 4))
        X = rng.standard_normal((n, d)).astype(np.float32)
        G = rng.integers(-1, n, size=(n, R)).astype(np.int32)
        for i in range(n):   # unique ids per row
            seen = set()
            for j in range(R):
                if G[i, j] in seen:
                    G[i, j] = -1
                seen.add(int(G[i, j]))
        entry = int(rng.integers(0, n))
        ix = _plain_index(X, G, entry)
        q = rng.standard_normal((1, d)).astype(np.float32)
        k = int(rng.integers(1, n + 1))
        r = oracle.search(ix, q, k, n, stage1=False, stage2_expansions=0, use_fes=False)
        reach, stack = {entry}, [entry]
        while stack:
            u = stack.pop()
            for v in G[u]:
                if v >= 0 and v not in reach:
                    reach.add(int(v))
                    stack.append(int(v))
        reach = np.array(sorted(reach))
        dd = ((q[0].astype(np.float64) - X[reach].astype(np.float64)) ** 2).sum(1).astype(np.float32)
        order = reach[np.lexsort((reach, dd))]
        exp = order[:k].tolist() + [-1] * (k - min(k, len(order)))
        assert r["ids"][0].tolist() == exp
        assert r["counters"][0, 4] == len(reach)          # every reachable node expanded once
        assert r["counters"][0, 5] == len(reach) - 1      # and its distance computed once


def test_ties_break_by_id():
    """Duplicated points tie exactly; the smaller id must come first."""
    X = np.asarray([[1.0, 0.0], [0.0, 0.0], [1.0, 0.0], [0.0, 0.0], [1.0, 0.0]], np.float32)
    G = np.asarray([[j for j in range(5) if j != i] for i in range(5)], np.int32)
    ix = _plain_index(X, G, 4)
    r = oracle.search(ix, np.asarray([[0.9, 0.0]], np.float32), 5, 5, stage1=False, stage2_expansions=0,
                      use_fes=False)
    assert r["ids"][0].tolist() == [0, 2, 4, 1, 3]


def test_dense_fes_is_argmin_over_entries(c1_small):
    """Table 2, 'FES (1 block)': dense FES is brute force over the entry set."""
    idx, Q, red32, _ = c1_small
    ix = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                            idx.full, idx.entry_ids, 0)
    _, qp = oracle.project(ix, Q)
    ent, dist = oracle.fes(ix, qp)
    sub_ids = np.nonzero(idx.subgraph_mask)[0]
    row_of = {int(v): i for i, v in enumerate(sub_ids)}
    E = np.asarray([red32[row_of[int(e)]] for e in idx.entry_ids], np.float64)
    for i in range(len(Q)):
        dd = ((qp[i].astype(np.float64) - E) ** 2).sum(1).astype(np.float32)
        j = np.lexsort((idx.entry_ids, dd))[0]
        assert ent[i] == idx.entry_ids[j]
        assert dist[i] == dd[j]


@pytest.mark.parametrize("T", [1, 3, 16])
@pytest.mark.parametrize("use_fes", [True, False])
def test_fes_seeds_are_the_best_entries(c1_small, T, use_fes):
    """Top-T seeding: stage (1) starts from the T entries closest to q' by
    (reduced FP32 distance, id) -- the first T of the entry set without FES --
    all of them visited.  With every stage off, C after stage (1) is exactly
    those seeds, checked here against a numpy brute force over the entries."""
    idx, Q, red32, _ = c1_small
    ix = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                            idx.full, idx.entry_ids, 0)
    r = oracle.search(ix, Q, 10, 64, stage1=False, stage2_expansions=0, stage3=False, use_fes=use_fes,
                      fes_seeds=T, pools=True)
    _, qp = oracle.project(ix, Q)
    sub_ids = np.nonzero(idx.subgraph_mask)[0]
    row_of = {int(v): i for i, v in enumerate(sub_ids)}
    ent = idx.entry_ids if use_fes else idx.entry_ids[:T]
    E = np.asarray([red32[row_of[int(e)]] for e in ent], np.float64)
    for i in range(len(Q)):
        dd = ((qp[i].astype(np.float64) - E) ** 2).sum(1).astype(np.float32)
        order = np.lexsort((ent, dd))[:T]
        assert r["pool1_ids"][i, :T].tolist() == ent[order].tolist()
        np.testing.assert_array_equal(r["pool1_dists"][i, :T], dd[order])
        assert np.all(r["pool1_ids"][i, T:] == -1)
        assert r["counters"][i, 7] == ent[order[0]]
    # with stage (1) on, every seed and every new stage-(1) distance is re-ranked (up to ef)
    r = oracle.search(ix, Q, 10, 64, use_fes=use_fes, fes_seeds=T)
    assert np.all(r["counters"][:, 6] == np.minimum(64, r["counters"][:, 1] + T))


def test_seeded_final_stage_hand_trace():
    """Sec. 4.2's experiment on the path graph: the final stage alone, seeded
    with given nodes (tests/golden/seeded_path_line.json)."""
    line = json.load(open(os.path.join(GOLDEN, "alg1_path_line.json")))
    g = json.load(open(os.path.join(GOLDEN, "seeded_path_line.json")))
    ix = _plain_index(line["points"], line["graph"], line["entry"])
    r = oracle.search(ix, np.asarray([line["query"]], np.float32), g["k"], g["ef"],
                      seed_ids=np.asarray([g["seeds"]], np.int32))
    assert r["ids"][0].tolist() == g["ids"]
    np.testing.assert_array_equal(r["dists"][0], np.asarray(g["dists"], np.float32))
    assert r["counters"][0].tolist() == g["counters"]


@pytest.mark.parametrize("metric", [0, 1])
def test_seeding_with_every_node_is_exact(metric):
    """Seeds = every node (ef >= N): each seed is scored once, no expansion
    finds an unvisited node, and the result is the exact top-k."""
    ix, X, rng = _exact_limit_index(40, 8, 6, 31, metric=metric, unit=(metric == 1))
    Q = rng.standard_normal((10, 8)).astype(np.float32)
    seeds = np.tile(rng.permutation(40).astype(np.int32), (len(Q), 1))
    r = oracle.search(ix, Q, 5, 40, seed_ids=seeds)
    gt, gd = oracle.bruteforce(X, Q, 5, metric=metric)
    assert np.array_equal(r["ids"], gt)
    assert np.all(r["counters"][:, 5] == 0) and np.all(r["counters"][:, 6] == 40)


def _with_clusters(idx, entry_cluster, centroids):
    return oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                              idx.full, idx.entry_ids, 0, np.asarray(entry_cluster, np.int32),
                              np.asarray(centroids, np.float32))


def test_clustered_fes_special_cases_equal_dense_fes(c1_small):
    """Sec. 5 / Table 2: with one cluster ('1 block') the clustered FES is the
    dense one; with one entry per cluster and each centroid equal to its
    entry's reduced row it again picks the dense argmin (entries are in
    ascending id order, so cluster-index ties break like id ties)."""
    idx, Q, red32, _ = c1_small
    sub_ids = np.nonzero(idx.subgraph_mask)[0]
    row_of = {int(v): i for i, v in enumerate(sub_ids)}
    E = np.asarray([red32[row_of[int(e)]] for e in idx.entry_ids], np.float32)
    dense = oracle.search(_with_clusters(idx, np.zeros(len(E)), E[:1]), Q, 10, 64, use_fes=True, fes_seeds=3)
    one = oracle.search(_with_clusters(idx, np.zeros(len(E)), E[:1]), Q, 10, 64, use_fes=2, fes_seeds=3)
    each = oracle.search(_with_clusters(idx, np.arange(len(E)), E), Q, 10, 64, use_fes=2)
    ref1 = oracle.search(_with_clusters(idx, np.zeros(len(E)), E[:1]), Q, 10, 64, use_fes=True)
    for a, b in ((one, dense), (each, ref1)):
        assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["counters"], b["counters"])


def test_clustered_fes_routes_then_takes_the_cluster_argmin(c1_small):
    """The entry is the (distance, id) argmin over the entries of the cluster
    whose centroid is closest to q' by (distance, cluster index)."""
    idx, Q, red32, _ = c1_small
    ix = _with_clusters(idx, idx.entry_cluster, idx.cluster_centroids)
    r = oracle.search(ix, Q, 10, 64, stage1=False, stage2_expansions=0, stage3=False, use_fes=2, pools=True)
    _, qp = oracle.project(ix, Q)
    sub_ids = np.nonzero(idx.subgraph_mask)[0]
    row_of = {int(v): i for i, v in enumerate(sub_ids)}
    E = np.asarray([red32[row_of[int(e)]] for e in idx.entry_ids], np.float64)
    C = idx.cluster_centroids.astype(np.float64)
    assert np.bincount(idx.entry_cluster).max() - np.bincount(idx.entry_cluster).min() <= 1
    for i in range(len(Q)):
        q = qp[i].astype(np.float64)
        dc = ((q - C) ** 2).sum(1).astype(np.float32)
        c = int(np.lexsort((np.arange(len(C)), dc))[0])
        members = np.nonzero(idx.entry_cluster == c)[0]
        dd = ((q - E[members]) ** 2).sum(1).astype(np.float32)
        j = members[np.lexsort((idx.entry_ids[members], dd))[0]]
        assert r["pool1_ids"][i, 0] == idx.entry_ids[j]


def test_graceful_degradation(c1_small):
    """Sec. 4.1 'Summary': with stages (1) and (2) off, the search is plain
    greedy search over the full graph from the FES entry.  With ef >= reach
    it is exact over the reachable set, whichever stages ran."""
    idx, Q, _, _ = c1_small
    ix = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                            idx.full, idx.entry_ids, 0)
    only3 = oracle.search(ix, Q[:8], 10, 64, stage1=False, stage2_expansions=0)
    assert np.all(only3["counters"][:, 0:4] == 0)
    staged = oracle.search(ix, Q[:8], 10, 64)
    gt, _ = oracle.bruteforce(idx.full, Q[:8], 10)
    assert oracle.recall_at_k(only3["ids"], gt, 10) > 0.9
    assert oracle.recall_at_k(staged["ids"], gt, 10) > 0.9


def test_stage2_runs_exactly_two_expansions(c1_small):
    idx, Q, _, _ = c1_small
    ix = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, 0, None,
                            idx.full, idx.entry_ids, 0)
    r = oracle.search(ix, Q, 10, 64)
    assert np.all(r["counters"][:, 2] == 2)
    assert np.all(r["counters"][:, 6] == np.minimum(64, r["counters"][:, 1] + 1))


def test_e4m3_and_bf16_decoders():
    """Format definitions, checked against hand values and torch's casts."""
    assert oracle.decode_e4m3(0x00) == 0.0
    assert oracle.decode_e4m3(0x01) == 2.0 ** -9          # smallest subnormal
    assert oracle.decode_e4m3(0x08) == 2.0 ** -6          # smallest normal
    assert oracle.decode_e4m3(0x38) == 1.0
    assert oracle.decode_e4m3(0x7E) == 448.0             # largest finite
    assert oracle.decode_e4m3(0xB8) == -1.0
    assert np.isnan(oracle.decode_e4m3(0x7F))
    codes = torch.arange(256, dtype=torch.uint8)
    ref = codes.view(torch.float8_e4m3fn).double().numpy()
    mine = np.array([oracle.decode_e4m3(c) for c in range(256)])
    assert np.array_equal(np.isnan(ref), np.isnan(mine))
    ok = ~np.isnan(ref)
    assert np.array_equal(ref[ok], mine[ok])
    rng = np.random.default_rng(0)
    vals = torch.from_numpy(rng.standard_normal(1000).astype(np.float32)).to(torch.bfloat16)
    bits = vals.view(torch.int16).numpy().view(np.uint16)
    assert all(oracle.decode_bf16(int(b)) == float(v) for b, v in zip(bits, vals.float()))


def test_recall_definition():
    found = np.asarray([[1, 2, 3], [4, 5, -1]])
    truth = np.asarray([[3, 2, 9], [5, 6, 7]])
    assert oracle.recall_at_k(found, truth, 3) == pytest.approx((2 + 1) / 6)


try:
    from hypothesis import given, settings, strategies as st
except ImportError:   # pragma: no cover
    given = None

if given is not None:
    @settings(max_examples=60, deadline=None)
    @given(st.integers(2, 20), st.integers(1, 4), st.integers(1, 3), st.integers(0, 2**31 - 1))
    def test_algorithm1_property_reachable_set(n, R, d, seed):
        """Algorithm 1 with ef >= N on any small graph (Sec. 2.2): the result is
        the brute-force top-k of the nodes reachable from the entry, every
        reachable node is expanded once, and each one but the entry has its
        distance computed once."""
        rng = np.random.default_rng(seed)
        X = rng.integers(-8, 9, size=(n, d)).astype(np.float32)   # small integers: exact FP32 distances
        G = np.full((n, R), -1, np.int32)
        for u in range(n):
            nb = rng.choice(n, size=min(R, n), replace=False)
            nb = nb[nb != u][: rng.integers(0, R + 1)]
            G[u, : len(nb)] = nb
        q = rng.integers(-8, 9, size=(1, d)).astype(np.float32)
        ix = _plain_index(X, G, 0)
        r = oracle.search(ix, q, min(3, n), n, stage1=False, stage2_expansions=0, use_fes=False)
        seen, stack = {0}, [0]
        while stack:
            u = stack.pop()
            for v in G[u]:
                if v >= 0 and int(v) not in seen:
                    seen.add(int(v))
                    stack.append(int(v))
        reach = np.asarray(sorted(seen))
        dd = ((X[reach].astype(np.float64) - q[0]) ** 2).sum(1).astype(np.float32)
        order = reach[np.lexsort((reach, dd))][: min(3, n)]
        got = r["ids"][0][r["ids"][0] >= 0]
        assert got.tolist() == order.tolist()
        assert r["counters"][0, 4] == len(reach)
        assert r["counters"][0, 5] == len(reach) - 1
