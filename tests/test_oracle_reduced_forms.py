"""Pins of the oracle's reduced-precision row path (Sec. 4.1 (1): stage (1)
reads x_primary; here stored as BF16, or as FP8 E4M3 codes times one FP32
scale per compact row).

Each check recomputes stage (1)'s distances with numpy in FP64 from the stored
codes, decoded independently of the oracle (BF16 by bit shift, FP8 through
torch's float8_e4m3fn cast), and compares them with the oracle's stage-(1)
candidate list element by element.  Inputs are dyadic rationals with few
significant bits, so every FP64 operation on both sides is exact and the one
rounding to FP32 is identical: any difference is a mistake, not rounding.

The sampled mask is a strict subset, so compact rows and original ids differ:
a scale or row taken by original id instead of compact row, a dropped scale,
or full rows used in place of reduced ones all change the candidate list."""
import json
import os

import numpy as np
import pytest
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _decode(codes, dtype, scales):
    if dtype == oracle.DTYPE_BF16:
        return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if dtype == oracle.DTYPE_FP8:
        x = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
        return x * scales.astype(np.float64)[:, None]
    return codes.astype(np.float64)


def _complete_subgraph(mask):
    """Every sampled node links to every other sampled node (-1 elsewhere)."""
    n = len(mask)
    ids = np.nonzero(mask)[0]
    sub = np.full((n, len(ids) - 1), -1, np.int32)
    for v in ids:
        sub[v] = [u for u in ids if u != v]
    return sub


def _random_case(dtype, seed, n=80, d=12):
    rng = np.random.default_rng(seed)
    mask = (rng.random(n) < 0.5).astype(np.uint8)
    mask[[3, 10]] = 1
    n_sub = int(mask.sum())
    # queries and full rows: multiples of 2^-5 in [-4, 4] (exact in every format used)
    X = (rng.integers(-128, 129, size=(n, d)) / 32.0).astype(np.float32)
    Q = (rng.integers(-128, 129, size=(6, d)) / 32.0).astype(np.float32)
    scales = None
    if dtype == oracle.DTYPE_BF16:
        vals = (rng.integers(-128, 129, size=(n_sub, d)) / 32.0).astype(np.float32)
        codes = (vals.view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal((codes.astype(np.uint32) << 16).view(np.float32), vals)
    else:
        # E4M3 normals with exponent field 4..10 (values 2^-3 .. 15), random sign
        e = rng.integers(4, 11, size=(n_sub, d))
        m = rng.integers(0, 8, size=(n_sub, d))
        s = rng.integers(0, 2, size=(n_sub, d))
        codes = ((s << 7) | (e << 3) | m).astype(np.uint8)
        # scales: multiples of 2^-8 in [0.5, 2], different per row
        scales = (rng.integers(128, 513, size=n_sub) / 256.0).astype(np.float32)
    G = np.stack([np.roll(np.arange(n), -j - 1) for j in range(4)], 1).astype(np.int32)   # a ring, for stage (3)
    entry = np.asarray([int(np.nonzero(mask)[0][0])], np.int32)
    return mask, codes, scales, X, Q, G, entry


@pytest.mark.parametrize("metric", [oracle.METRIC_L2, oracle.METRIC_IP])
@pytest.mark.parametrize("dtype", [oracle.DTYPE_BF16, oracle.DTYPE_FP8])
def test_stage1_pool_is_the_bruteforce_of_the_decoded_rows(dtype, metric):
    """Complete subgraph among the sampled nodes, d' = d, ef >= N: stage (1)
    scores every sampled node, so its candidate list is the exact (distance,
    id) order of all of them under the decoded reduced rows."""
    for seed in range(4):
        mask, codes, scales, X, Q, G, entry = _random_case(dtype, 100 * dtype + 10 * metric + seed)
        n, d = X.shape
        ix = oracle.OracleIndex(G, mask, _complete_subgraph(mask), np.eye(d), codes, dtype, scales, X, entry, metric)
        r = oracle.search(ix, Q, 5, n, stage2_expansions=0, stage3=False, pools=True)
        ids = np.nonzero(mask)[0]
        R = _decode(codes, dtype, scales)
        for i, q in enumerate(Q.astype(np.float64)):
            dd = ((q - R) ** 2).sum(1) if metric == oracle.METRIC_L2 else -(R @ q)
            d32 = dd.astype(np.float32)
            order = np.lexsort((ids, d32))
            assert r["pool1_ids"][i, :len(ids)].tolist() == ids[order].tolist(), (seed, i)
            np.testing.assert_array_equal(r["pool1_dists"][i, :len(ids)], d32[order])
            assert np.all(r["pool1_ids"][i, len(ids):] == -1)
            assert r["counters"][i, 0] == len(ids) and r["counters"][i, 1] == len(ids) - 1


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_fp8_scale_hand_trace(metric):
    """tests/golden/fp8_scales_2d.json: two rows with equal codes and
    different scales; the order is derived by hand."""
    g = json.load(open(os.path.join(GOLDEN, "fp8_scales_2d.json")))
    n = g["n"]
    mask = np.asarray(g["mask"], np.uint8)
    sub = np.full((n, 3), -1, np.int32)
    for v, row in g["subgraph_rows"].items():
        sub[int(v)] = row
    codes = np.asarray(g["codes"], np.uint8)
    scales = np.asarray(g["scales"], np.float32)
    X = np.zeros((n, 2), np.float32)
    X[np.nonzero(mask)[0]] = _decode(codes, oracle.DTYPE_FP8, scales)
    G = sub.copy()
    m = oracle.METRIC_L2 if metric == "l2" else oracle.METRIC_IP
    ix = oracle.OracleIndex(G, mask, sub, np.eye(2), codes, oracle.DTYPE_FP8, scales, X,
                            np.asarray([g["entry"]], np.int32), m)
    r = oracle.search(ix, np.asarray([g["query"]], np.float32), 2, g["ef"], stage2_expansions=0, stage3=False,
                      pools=True)
    exp = g[metric]
    assert r["pool1_ids"][0].tolist() == exp["pool1"]
    np.testing.assert_array_equal(r["pool1_dists"][0], np.asarray(exp["pool1_dists"], np.float32))
    assert r["counters"][0, 0] == exp["exp1"] and r["counters"][0, 1] == exp["dist1"]
    assert r["counters"][0, 7] == g["entry"]


@pytest.mark.parametrize("dtype", [oracle.DTYPE_BF16, oracle.DTYPE_FP8])
def test_fes_reads_the_decoded_entry_rows(dtype):
    """Dense FES (Sec. 5) over entries stored in a reduced format: the entry
    is the (distance, id) argmin under the decoded rows."""
    mask, codes, scales, X, Q, G, _ = _random_case(dtype, 7 + dtype)
    n, d = X.shape
    ids = np.nonzero(mask)[0]
    entries = ids[1::2].astype(np.int32)
    ix = oracle.OracleIndex(G, mask, _complete_subgraph(mask), np.eye(d), codes, dtype, scales, X, entries,
                            oracle.METRIC_L2)
    ent, dist = oracle.fes(ix, Q)
    R = _decode(codes, dtype, scales)
    rows = np.searchsorted(ids, entries)
    for i, q in enumerate(Q.astype(np.float64)):
        d32 = ((q - R[rows]) ** 2).sum(1).astype(np.float32)
        j = np.lexsort((entries, d32))[0]
        assert ent[i] == entries[j] and dist[i] == d32[j]
