"""The autotuner (pilot_autotune) through the C ABI: it only changes the
search kernel's launch shape, so results stay identical to the oracle; the
shape it picks applies to later automatic searches and servers; the cache
file round-trips."""
import os

import numpy as np
import pytest

import oracle
from paper_2503_21206_b300 import index_build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21206_b300 import build
    build.build()
    from paper_2503_21206_b300 import pilot
    w = synth.WORKLOADS["c1_mixture_20k_d96"]
    idx, Q, _, _ = index_build.build_workload(w, n=6000, nq=120)
    return pilot, idx, Q


def _oracle(idx, Q, k, ef):
    oi = oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, oracle.DTYPE_F32,
                            idx.reduced_scales, idx.full, idx.entry_ids, idx.metric)
    return oracle.search(oi, Q, k, ef)


def test_tuned_shape_keeps_results(env):
    pilot, idx, Q = env
    g = pilot.load_index_data(idx)
    r = pilot.pilot_autotune(g, Q, 10, 64)
    assert r["from_cache"] == 0 and r["candidates"] >= 1
    assert 1 <= r["warps_per_block"] <= 8 and r["stage_rows"] in (0, 4, 8, 12, 16, 20, 24, 32)
    assert 0 < r["best_ms"] <= r["default_ms"]
    ref = _oracle(idx, Q, 10, 64)
    ids, d = pilot.pilot_search(g, Q, 10, 64)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(d, ref["dists"])


def test_other_ef_classes_untouched_and_explicit_options_win(env):
    pilot, idx, Q = env
    g = pilot.load_index_data(idx)
    pilot.pilot_autotune(g, Q[:40], 10, 200)          # class 256
    ref = _oracle(idx, Q[:40], 10, 40)                 # class 64: defaults
    ids, d = pilot.pilot_search(g, Q[:40], 10, 40)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(d, ref["dists"])
    o = pilot.pilot_search_options_default()
    o.warps_per_block, o.stage_rows = 1, 8
    ref = _oracle(idx, Q[:40], 10, 200)
    ids, d = pilot.pilot_search_ex(g, Q[:40], 10, 200, options=o)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(d, ref["dists"])


def test_cache_round_trip(env, tmp_path):
    pilot, idx, Q = env
    cache = str(tmp_path / "tune.txt")
    g1 = pilot.load_index_data(idx)
    a = pilot.pilot_autotune(g1, Q, 10, 96, cache_path=cache)
    assert a["from_cache"] == 0 and os.path.getsize(cache) > 0
    line = open(cache).read().strip().split()
    assert len(line) == 4 and int(line[1]) == a["warps_per_block"] and int(line[2]) == a["stage_rows"]
    g2 = pilot.load_index_data(idx)
    b = pilot.pilot_autotune(g2, Q, 10, 128, cache_path=cache)   # same class (2^7)
    assert b["from_cache"] == 1 and b["candidates"] == 0
    assert (b["warps_per_block"], b["stage_rows"]) == (a["warps_per_block"], a["stage_rows"])
    c = pilot.pilot_autotune(g2, Q[:20], 10, 300, cache_path=cache)   # another class: timed, appended
    assert c["from_cache"] == 0 and len(open(cache).read().strip().split("\n")) == 2


def test_server_after_tuning_matches_search(env):
    pilot, idx, Q = env
    g = pilot.load_index_data(idx)
    pilot.pilot_autotune(g, Q, 10, 128)
    srv = pilot.pilot_serve_create(g, max_ef=128, max_k=10, expansions_per_step=8)
    try:
        tickets = [srv.submit(Q[i], 10, 100) for i in range(32)]
        for i, t in enumerate(tickets):
            ids, d = srv.wait(t, 10)
            ref_ids, ref_d = pilot.pilot_search(g, np.ascontiguousarray(Q[i:i + 1]), 10, 100)
            assert np.array_equal(ids, ref_ids[0]) and np.array_equal(d, ref_d[0])
    finally:
        srv.destroy()


def test_rejects_bad_arguments(env):
    pilot, idx, Q = env
    g = pilot.load_index_data(idx)
    with pytest.raises(pilot.PilotError):
        pilot.pilot_autotune(g, Q[:0], 10, 64)
    with pytest.raises(pilot.PilotError):
        pilot.pilot_autotune(g, Q, 10, 5)
    with pytest.raises(pilot.PilotError):
        pilot.pilot_autotune(g, Q, 10, 1024)


def test_stage_switches_are_part_of_the_key(env, tmp_path):
    pilot, idx, Q = env
    cache = str(tmp_path / "tune.txt")
    g = pilot.load_index_data(idx)
    plain = pilot.pilot_search_options_default()
    plain.stage1, plain.stage2_expansions = 0, 0
    a = pilot.pilot_autotune(g, Q[:40], 10, 64, options=plain, cache_path=cache)
    b = pilot.pilot_autotune(g, Q[:40], 10, 64, cache_path=cache)
    assert a["from_cache"] == 0 and b["from_cache"] == 0
    keys = [ln.split()[0] for ln in open(cache).read().strip().split("\n")]
    assert len(keys) == 2 and keys[0] != keys[1] and keys[0].endswith("|s0.0.1.1") and keys[1].endswith("|s1.2.1.1")
    ref = _oracle(idx, Q[:40], 10, 64)
    ids, d = pilot.pilot_search(g, Q[:40], 10, 64)
    assert np.array_equal(ids, ref["ids"]) and np.array_equal(d, ref["dists"])
