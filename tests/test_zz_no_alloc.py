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
    # at d = 96 a query takes 96*4 (padded row) + 64*4 + 64*2 (projection, FP32
    # and BF16) + 16*4 (FES candidates) + 8 + 4 = 844 bytes of scratch, so about
    # 19,900 queries fit in the 16 MiB array; 40,000 do not
    nq = 40_000
    q = torch.zeros((nq, Q.shape[1]), dtype=torch.float32, device="cuda")
    ids, d = _device_out(torch, nq, 10)
    with pytest.raises(pilot.PilotError) as e:
        pilot.pilot_search_noalloc(g, q, 10, 64, ids, d)
    assert e.value.status == pilot.PILOT_EINVAL and "split the batch" in str(e.value)


def test_rejects_host_buffers(setup):
    torch, pilot, g, Q = setup
    q = np.ascontiguousarray(Q[:4])
    ids = np.empty((4, 10), np.int32)
    d = np.empty((4, 10), np.float32)
    # the binding refuses before any pointer reaches the library ...
    with pytest.raises(ValueError):
        pilot.pilot_search_noalloc(g, q, 10, 64, ids, d)
    # ... and the C entry point itself rejects host memory
    rc = pilot._lib.pilot_search_noalloc(g.handle, q.ctypes.data, 4, 10, 64, ids.ctypes.data, d.ctypes.data, None)
    assert rc == pilot.PILOT_EINVAL and "device-resident" in pilot.pilot_last_error()


def test_calls_allocate_no_device_memory(setup):
    """The property the entry point exists for: once the library's kernels are
    loaded, calls leave the device's free memory unchanged, even for a batch
    larger than any the index has seen (a workspace that grows would show)."""
    torch, pilot, _, Q = setup
    from paper_2503_21206_b300 import index_build, synth
    w = synth.WORKLOADS["c1_mixture_20k_d96"]
    idx, _, _, _ = index_build.build_workload(w, n=3000, nq=8)
    g = pilot.load_index_data(idx)          # a fresh index: its search workspace is empty
    big = 5000
    q = torch.from_numpy(np.ascontiguousarray(np.resize(Q, (big, Q.shape[1])))).cuda()
    ids, d = _device_out(torch, big, 10)
    pilot.pilot_search_noalloc(g, q[:64], 10, 64, ids, d)   # loads the kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        pilot.pilot_search_noalloc(g, q, 10, 64, ids, d)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref_ids, _ = pilot.pilot_search(g, q.cpu().numpy(), 10, 64)
    assert np.array_equal(ids.cpu().numpy(), ref_ids)
    g.free()
