"""pilot_search_noalloc: the search entry point for callers that cannot let the
library allocate device memory during a call (callers whose memory belongs to
their own pool or allocator, or that cannot pay an allocation's
synchronisation).  Its results must equal pilot_search's on the same inputs,
call after call, although every call reuses one fixed scratch array.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_21206_b300 import build, index_build, synth
    build.build()
    from paper_2503_21206_b300 import pilot
    w = synth.WORKLOADS["c1_mixture_20k_d96"]
    idx, Q, _, _ = index_build.build_workload(w, n=4000, nq=300)
    return torch, pilot, pilot.load_index_data(idx), Q


def _device_out(torch, nq, k):
    return (torch.full((nq, k), -7, dtype=torch.int32, device="cuda"),
            torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda"))


def test_two_calls_in_a_row_match_pilot_search(setup):
    torch, pilot, g, Q = setup
    # two different batches back to back: the second call runs on the scratch
    # the first one left behind
    for rows, k, ef in ((slice(0, 300), 10, 64), (slice(17, 150), 5, 96)):
        q = torch.from_numpy(np.ascontiguousarray(Q[rows])).cuda()
        ref_ids, ref_d = pilot.pilot_search(g, q.cpu().numpy(), k, ef)
        ids, d = _device_out(torch, q.shape[0], k)
        pilot.pilot_search_noalloc(g, q, k, ef, ids, d)
        torch.cuda.synchronize()
        assert np.array_equal(ids.cpu().numpy(), ref_ids)
        assert np.array_equal(d.cpu().numpy(), ref_d)


def test_rejects_a_batch_larger_than_the_scratch(setup):
    torch, pilot, g, Q = setup
    nq = 40_000   # ~700 bytes of scratch each at d = 96: beyond the fixed array
    q = torch.zeros((nq, Q.shape[1]), dtype=torch.float32, device="cuda")
    ids, d = _device_out(torch, nq, 10)
    with pytest.raises(pilot.PilotError) as e:
        pilot.pilot_search_noalloc(g, q, 10, 64, ids, d)
    assert e.value.status == pilot.PILOT_EINVAL and "split the batch" in str(e.value)


def test_rejects_host_buffers(setup):
    torch, pilot, g, Q = setup
    ids = np.empty((4, 10), np.int32)
    d = np.empty((4, 10), np.float32)
    with pytest.raises(pilot.PilotError) as e:
        pilot.pilot_search_noalloc(g, np.ascontiguousarray(Q[:4]), 10, 64, ids, d)
    assert e.value.status == pilot.PILOT_EINVAL
