"""The offline input step: graph, subgraph, SVD rows, quantisation, files."""
import numpy as np
import pytest
import torch

from paper_2503_21206_b300 import index_build, synth


def _reach(adj, sources):
    return index_build._reached_from(adj, np.asarray(sources))


def test_graph_well_formed(c1_small):
    idx, _, _, _ = c1_small
    n = idx.n
    for G, rows in ((idx.graph, np.arange(n)), (idx.subgraph, np.nonzero(idx.subgraph_mask)[0])):
        sub = G[rows]
        assert sub.min() >= -1 and sub.max() < n
        assert np.all((sub >= 0).sum(1) >= 1)
        for r, row in zip(rows, sub):
            v = row[row >= 0]
            assert len(set(v.tolist())) == len(v)
            assert r not in v
    # unsampled nodes keep zero out-degree and receive no subgraph edge (Sec. 4.3)
    assert np.all(idx.subgraph[idx.subgraph_mask == 0] == -1)
    tgt = idx.subgraph[idx.subgraph >= 0]
    assert np.all(idx.subgraph_mask[tgt] == 1)
    # every node is reachable from the entry set in the full graph, and every
    # sampled node in the subgraph
    assert _reach(idx.graph, idx.entry_ids).all()
    r = _reach(idx.subgraph, idx.entry_ids)
    assert np.array_equal(r, idx.subgraph_mask == 1)
    assert np.all(idx.subgraph_mask[idx.entry_ids] == 1)


def test_reduced_rows_are_projected_sampled_rows(c1_small):
    idx, _, red32, V = c1_small
    sampled = np.nonzero(idx.subgraph_mask)[0]
    ref = (idx.full[sampled].astype(np.float64) @ V[:, :idx.dp]).astype(np.float32)
    assert np.array_equal(red32, ref)
    assert np.array_equal(idx.reduced, red32)


def test_quantisation_formats():
    rng = np.random.default_rng(1)
    red = rng.standard_normal((50, 32)).astype(np.float32)
    red[3] = 0.0
    b, _ = index_build.quantize_rows(red, "bf16")
    ref = torch.from_numpy(red).to(torch.bfloat16).float().numpy()
    back = (b.astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(back, ref)
    c, s = index_build.quantize_rows(red, "fp8")
    assert s[3] == 1.0 and np.all(c[3] == 0)
    deq = torch.from_numpy(c).view(torch.float8_e4m3fn).float().numpy() * s[:, None]
    err = np.abs(deq - red)
    assert np.all(err <= np.abs(red) * 2.0 ** -4 + s[:, None] * 2.0 ** -9 + 1e-30)
    assert np.all(np.abs(c.view(np.uint8) & 0x7F) <= 0x7E)   # no NaN codes


def test_save_load_roundtrip(tmp_path, c1_small):
    idx, _, _, _ = c1_small
    index_build.save_index(idx, str(tmp_path))
    back = index_build.load_index(str(tmp_path))
    for name in ("graph", "subgraph_mask", "subgraph", "basis", "reduced", "full", "entry_ids"):
        assert np.array_equal(getattr(idx, name), getattr(back, name))
    assert back.metric == idx.metric and back.reduced_dtype == idx.reduced_dtype


def test_exact_topk_matches_bruteforce(c1_small):
    import oracle
    idx, Q, _, _ = c1_small
    a, _ = index_build.exact_topk(idx.full, Q, 10)
    b, _ = oracle.bruteforce(idx.full, Q, 10)
    assert np.array_equal(a, b)


def test_workloads_are_seeded_and_prefix_stable():
    w = synth.WORKLOADS["c2_aniso_1m_d96"]
    x1, q1 = synth.generate(w, n=500, nq=10)
    x2, q2 = synth.generate(w, n=500, nq=10)
    assert np.array_equal(x1, x2) and np.array_equal(q1, q2)
    np.testing.assert_allclose(np.linalg.norm(x1, axis=1), 1.0, rtol=1e-5)
    for name in ("c1_mixture_20k_d96", "c2_aniso_1m_d96"):
        wl = synth.WORKLOADS[name]
        xa, qa = synth.generate(wl, n=300, nq=20)
        xb, qb = synth.generate(wl, n=900, nq=70)
        assert np.array_equal(xa, xb[:300]) and np.array_equal(qa, qb[:20])


def test_entry_clusters_are_bucket_aligned_and_seeded():
    """The clustered FES's coarse clusters (Sec. 5): non-empty clusters of at
    most ceil(n / r) entries (exactly n / r each when r divides n), each
    centroid the mean of its members, the same assignment for the same seed."""
    rng = np.random.default_rng(3)
    E = rng.standard_normal((1000, 16)).astype(np.float32)
    a1, c1 = index_build.cluster_entries(E, 32, 9)
    a2, c2 = index_build.cluster_entries(E, 32, 9)
    assert np.array_equal(a1, a2) and np.array_equal(c1, c2)
    sizes = np.bincount(a1, minlength=32)
    assert c1.shape == (32, 16) and sizes.min() >= 1 and sizes.max() <= 32
    even, _ = index_build.cluster_entries(E[:992], 32, 9)
    assert np.all(np.bincount(even, minlength=32) == 31)
    for c in range(32):
        np.testing.assert_allclose(c1[c], E[a1 == c].astype(np.float64).mean(0), rtol=1e-5, atol=1e-6)
    a3, c3 = index_build.cluster_entries(E[:5], 32, 9)      # fewer entries than clusters: one each
    assert sorted(a3.tolist()) == list(range(5)) and c3.shape == (5, 16)


def test_save_load_keeps_entry_clusters(tmp_path, c1_small):
    idx, _, _, _ = c1_small
    index_build.save_index(idx, str(tmp_path))
    back = index_build.load_index(str(tmp_path))
    assert np.array_equal(back.entry_cluster, idx.entry_cluster)
    assert np.array_equal(back.cluster_centroids, idx.cluster_centroids)


def test_ivf_candidates_are_exact_sorted_and_mostly_the_nearest():
    """Inverted-list candidates (for base sets too large for the exact
    search): every candidate's distance is its exact FP32 squared distance,
    a row never lists itself, rows are in (distance, id) order, and on a
    well-separated mixture most true nearest neighbours are found."""
    rng = np.random.default_rng(4)
    centres = rng.standard_normal((40, 16)) * 8.0
    X = (centres[rng.integers(0, 40, 6000)] + 0.5 * rng.standard_normal((6000, 16))).astype(np.float32)
    ids, dst = index_build.ivf_candidates(X, 12, nlist=24, nprobe=4, seed=3)
    ids, dst = ids.numpy(), dst.numpy()
    ex_ids, _ = index_build.knn_candidates(X, 12)
    ex_ids = ex_ids.numpy()
    for i in rng.integers(0, 6000, 200):
        c = ids[i][ids[i] >= 0]
        d = ((X[i].astype(np.float64) - X[c].astype(np.float64)) ** 2).sum(1)
        np.testing.assert_allclose(dst[i][:len(c)], d, rtol=2e-6)
        assert i not in c
        key = list(zip(dst[i][:len(c)].tolist(), c.tolist()))
        assert key == sorted(key)
    recall = np.mean([len(set(a) & set(b)) / 12 for a, b in zip(ids, ex_ids)])
    assert recall > 0.95, recall
