"""Serving (continuous batching) through the C ABI, checked against the CPU
oracle: every served request returns the oracle's staged search (Sec. 4.1)
for its own query, k and ef -- ids, distances and per-stage counters --
whether it ran alone or in a mix of k and ef with requests arriving while
others are on the GPU.  Also admission limits, queueing, timeouts and
statistics."""
import os
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2503_21206_b300 import index_build, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def _oracle_index(idx):
    dt = {"f32": oracle.DTYPE_F32, "bf16": oracle.DTYPE_BF16, "fp8": oracle.DTYPE_FP8}[idx.reduced_dtype]
    return oracle.OracleIndex(idx.graph, idx.subgraph_mask, idx.subgraph, idx.basis, idx.reduced, dt,
                              idx.reduced_scales, idx.full, idx.entry_ids, idx.metric)


def _oracle_answers(oi, Q, rows, ks, efs):
    """Oracle result (ids, dists, counters) of every request, grouped by (k, ef)."""
    out = [None] * len(rows)
    groups = {}
    for j, (k, ef) in enumerate(zip(ks, efs)):
        groups.setdefault((int(k), int(ef)), []).append(j)
    for (k, ef), js in groups.items():
        r = oracle.search(oi, Q[[rows[j] for j in js]], k, ef, nthreads=THREADS)
        for i, j in enumerate(js):
            out[j] = (r["ids"][i], r["dists"][i], r["counters"][i])
    return out


def _assert_same(got, ref, what):
    ids, d, cnt = got
    rid, rd, rc = ref
    assert np.array_equal(ids, rid), (what, ids, rid)
    assert np.array_equal(d, rd), (what, d, rd)
    assert np.array_equal(cnt, rc), (what, cnt, rc)


@pytest.fixture(scope="module", params=["f32_d96", "bf16_d256"])
def env(request):
    """A C1-shaped FP32 index (d = 96, d' = 32) and a C4-shaped one (Gaussian
    mixture, d = 256, d' = 64 BF16 rows, 20% subgraph)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21206_b300 import build
    build.build()
    from paper_2503_21206_b300 import pilot
    if request.param == "f32_d96":
        idx, Q, _, _ = index_build.build_workload(synth.WORKLOADS["c1_mixture_20k_d96"], n=8000, nq=160)
    else:
        idx, Q, _, _ = index_build.build_workload(synth.WORKLOADS["c4_mixture_10m_d256"], n=12000, nq=160,
                                                  reduced_dtype="bf16")
    assert idx.reduced_dtype == request.param.split("_")[0]
    return pilot, pilot.load_index_data(idx), Q, _oracle_index(idx)


def test_mixed_k_and_ef_with_arrivals_equal_the_oracle(env):
    """k from {1, 10, 100}, ef uniform in [max(32, k), 512]; waves submitted
    from another thread while earlier requests are in flight (a small step
    budget keeps every request resident for many steps)."""
    pilot, g, Q, oi = env
    rng = np.random.default_rng(11)
    n_req = 120
    rows = rng.integers(0, len(Q), n_req)
    ks = rng.choice([1, 10, 100], size=n_req)
    efs = np.array([int(rng.integers(max(32, k), 513)) for k in ks])
    ref = _oracle_answers(oi, Q, rows, ks, efs)
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=100, expansions_per_step=24, max_slots=48)
    tickets = {}

    def producer():
        for wave in range(6):
            for j in range(wave * 20, wave * 20 + 20):
                tickets[j] = srv.submit(Q[rows[j]], int(ks[j]), int(efs[j]))
            time.sleep(0.003)

    try:
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for j in range(n_req):
            _assert_same(srv.wait(tickets[j], int(ks[j]), counters=True), ref[j], j)
        st = srv.stats()
        assert st["completed"] == n_req and st["admitted"] == n_req
        assert st["steps"] > 10 and 0 < st["p50_ms"] <= st["p99_ms"] and st["qps"] > 0
        assert st["visited_overflows"] == 0
    finally:
        srv.destroy()
    # the same requests one at a time: each result is the same alone as in the mix
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=100, expansions_per_step=24, max_slots=48)
    try:
        for j in range(0, n_req, 15):
            t = srv.submit(Q[rows[j]], int(ks[j]), int(efs[j]))
            _assert_same(srv.wait(t, int(ks[j]), counters=True), ref[j], ("alone", j))
    finally:
        srv.destroy()


def test_submit_batch_equals_the_oracle(env):
    """Requests queued with one pilot_serve_submit_batch call (mixed k and ef)
    return the oracle's results; a batch with one bad request queues nothing."""
    pilot, g, Q, oi = env
    rng = np.random.default_rng(23)
    n_req = 64
    rows = rng.integers(0, len(Q), n_req)
    ks = rng.choice([1, 10, 100], size=n_req).astype(np.int32)
    efs = np.array([int(rng.integers(max(32, k), 513)) for k in ks], np.int32)
    ref = _oracle_answers(oi, Q, rows, ks, efs)
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=100)
    try:
        bad_ef = efs.copy()
        bad_ef[5] = 600
        with pytest.raises(pilot.PilotError) as e:
            srv.submit_batch(Q[rows], ks, bad_ef)
        assert e.value.status == pilot.PILOT_EINVAL
        assert srv.stats()["submitted"] == 0
        tickets = srv.submit_batch(Q[rows], ks, efs)
        assert len(set(tickets.tolist())) == n_req
        for j in range(n_req):
            _assert_same(srv.wait(int(tickets[j]), int(ks[j]), counters=True), ref[j], j)
        assert srv.stats()["completed"] == n_req
    finally:
        srv.destroy()


def test_batch_search_equals_the_oracle_at_serving_shapes(env):
    """The batch entry point on the same index and (k, ef) mix, for reference."""
    pilot, g, Q, oi = env
    for k, ef in ((1, 32), (10, 200), (100, 512)):
        cnt = np.empty((40, 8), np.int32)
        ids, d = pilot.pilot_search_ex(g, np.ascontiguousarray(Q[:40]), k, ef, counters=cnt)
        r = oracle.search(oi, Q[:40], k, ef, nthreads=THREADS)
        assert np.array_equal(ids, r["ids"]) and np.array_equal(d, r["dists"])
        assert np.array_equal(cnt, r["counters"])


def test_admission_limits(env):
    pilot, g, Q, oi = env
    ref = oracle.search(oi, Q, 10, 64, nthreads=THREADS)
    srv = pilot.pilot_serve_create(g, max_ef=64, max_k=10, queue_capacity=4, max_slots=2, expansions_per_step=1)
    try:
        with pytest.raises(pilot.PilotError) as e:
            srv.submit(Q[0], 10, 65)       # above the shared-memory budget of the step kernel
        assert e.value.status == pilot.PILOT_EINVAL
        with pytest.raises(pilot.PilotError) as e:
            srv.submit(Q[0], 11, 64)
        assert e.value.status == pilot.PILOT_EINVAL
        bad = Q[0].copy()
        bad[3] = np.inf
        with pytest.raises(pilot.PilotError) as e:
            srv.submit(bad, 10, 64)
        assert e.value.status == pilot.PILOT_EINVAL
        tickets, busy = [], 0
        for i in range(200):
            try:
                tickets.append((i, srv.submit(Q[i % len(Q)], 10, 64)))
            except pilot.PilotError as err:
                assert err.status == pilot.PILOT_EBUSY
                busy += 1
        assert busy > 0
        for i, t in tickets:
            ids, d = srv.wait(t, 10)
            assert np.array_equal(ids, ref["ids"][i % len(Q)]) and np.array_equal(d, ref["dists"][i % len(Q)])
        assert srv.stats()["rejected"] == busy
    finally:
        srv.destroy()


def test_wait_timeout_keeps_ticket(env):
    pilot, g, Q, oi = env
    ref = oracle.search(oi, Q[:3], 10, 512, nthreads=THREADS)
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=10, expansions_per_step=1, max_slots=1)
    try:
        tickets = [srv.submit(Q[i], 10, 512) for i in range(3)]
        with pytest.raises(pilot.PilotError) as e:
            srv.wait(tickets[-1], 10, timeout_ms=0)
        assert e.value.status == pilot.PILOT_ETIMEOUT
        for i, t in enumerate(tickets):
            _assert_same(srv.wait(t, 10, counters=True), (ref["ids"][i], ref["dists"][i], ref["counters"][i]), i)
        with pytest.raises(pilot.PilotError):
            srv.wait(tickets[0], 10, timeout_ms=0)      # collected already: unknown now -> timeout or invalid
    finally:
        srv.destroy()


def test_step_timeout_fails_the_waiters(env):
    """A bounded host wait that runs out: with step_timeout_ms = 1 a step that
    takes longer fails the server, every waiter gets PILOT_ETIMEOUT (or its
    result, if it finished first) and new work is refused.  The kernel itself
    runs to completion, so the GPU stays usable."""
    pilot, g, Q, _ = env
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=10, expansions_per_step=1 << 20, step_timeout_ms=1)
    try:
        tickets, refused = [], None
        for i in range(3000):
            try:
                tickets.append(srv.submit(Q[i % len(Q)], 10, 512))
            except pilot.PilotError as e:   # a step already timed out: the server refuses new work
                refused = e.status
                break
        assert refused in (None, pilot.PILOT_ETIMEOUT)
        codes = []
        for t in tickets:
            try:
                srv.wait(t, 10, timeout_ms=60_000)
                codes.append(pilot.PILOT_OK)
            except pilot.PilotError as e:
                codes.append(e.status)
        assert pilot.PILOT_ETIMEOUT in codes or refused == pilot.PILOT_ETIMEOUT
        assert set(codes) <= {pilot.PILOT_OK, pilot.PILOT_ETIMEOUT}
        with pytest.raises(pilot.PilotError) as e:
            srv.submit(Q[0], 10, 64)
        assert e.value.status == pilot.PILOT_ETIMEOUT
    finally:
        srv.destroy()
    # the device is still usable afterwards
    ids, _ = pilot.pilot_search(g, np.ascontiguousarray(Q[:4]), 10, 64)
    assert ids.shape == (4, 10) and (ids >= 0).all()
