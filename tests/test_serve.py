"""Serving (continuous batching) through the C ABI: each result equals the
batch search of that query alone, whether it ran alone or in a mix of k and
ef with requests arriving while others are on the GPU; admission limits,
queueing, timeouts and statistics."""
import threading
import time

import numpy as np
import pytest

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
    idx, Q, _, _ = index_build.build_workload(w, n=8000, nq=160)
    return pilot, pilot.load_index_data(idx), Q


def _alone(pilot, g, q, k, ef):
    ids, d = pilot.pilot_search(g, np.ascontiguousarray(q[None, :]), k, ef)
    return ids[0], d[0]


def test_results_in_a_mix_equal_results_alone(env):
    pilot, g, Q = env
    rng = np.random.default_rng(7)
    ks = rng.choice([1, 10, 50], size=len(Q))
    efs = np.array([int(rng.integers(k, 129)) for k in ks])
    srv = pilot.pilot_serve_create(g, max_ef=128, max_k=50, expansions_per_step=8)
    try:
        tickets = [srv.submit(Q[i], int(ks[i]), int(efs[i])) for i in range(len(Q))]
        for i, t in enumerate(tickets):
            ids, d = srv.wait(t, int(ks[i]))
            ref_ids, ref_d = _alone(pilot, g, Q[i], int(ks[i]), int(efs[i]))
            assert np.array_equal(ids, ref_ids), i
            assert np.array_equal(d, ref_d), i
        st = srv.stats()
        assert st["completed"] == len(Q) and st["admitted"] == len(Q)
        assert st["steps"] > 1 and 0 < st["p50_ms"] <= st["p99_ms"] and st["qps"] > 0
    finally:
        srv.destroy()


def test_arrivals_while_others_run(env):
    """Waves submitted from another thread while earlier requests are in
    flight join at later steps; every result still equals the search alone."""
    pilot, g, Q = env
    srv = pilot.pilot_serve_create(g, max_ef=64, max_k=10, expansions_per_step=4, max_slots=32)
    out = {}

    def producer():
        for wave in range(4):
            for i in range(wave * 40, wave * 40 + 40):
                out[i] = srv.submit(Q[i], 10, 64)
            time.sleep(0.002)

    try:
        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for i, t in out.items():
            ids, d = srv.wait(t, 10)
            ref_ids, ref_d = _alone(pilot, g, Q[i], 10, 64)
            assert np.array_equal(ids, ref_ids) and np.array_equal(d, ref_d), i
        st = srv.stats()
        assert st["slots"] == 32 and st["completed"] == 160
    finally:
        srv.destroy()


def test_admission_limits(env):
    pilot, g, Q = env
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
            assert np.array_equal(ids, _alone(pilot, g, Q[i % len(Q)], 10, 64)[0])
        assert srv.stats()["rejected"] == busy
    finally:
        srv.destroy()


def test_wait_timeout_keeps_ticket(env):
    pilot, g, Q = env
    srv = pilot.pilot_serve_create(g, max_ef=512, max_k=10, expansions_per_step=1, max_slots=1)
    try:
        tickets = [srv.submit(Q[i], 10, 512) for i in range(3)]
        with pytest.raises(pilot.PilotError) as e:
            srv.wait(tickets[-1], 10, timeout_ms=0)
        assert e.value.status == pilot.PILOT_ETIMEOUT
        for i, t in enumerate(tickets):
            ids, _ = srv.wait(t, 10)
            assert np.array_equal(ids, _alone(pilot, g, Q[i], 10, 512)[0])
        with pytest.raises(pilot.PilotError):
            srv.wait(tickets[0], 10, timeout_ms=0)      # collected already: unknown now -> timeout or invalid
    finally:
        srv.destroy()
