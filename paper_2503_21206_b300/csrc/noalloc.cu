// noalloc.cu -- pilot_search_noalloc: a search entry point that allocates
// nothing.
//
// pilot_search keeps per-call scratch (padded queries, projected queries, FES
// candidates, status words) in a workspace it grows with cudaMalloc.  Some
// callers cannot allow that: code running inside a custom allocator or a
// memory pool that must own every device allocation, real-time loops where an
// allocation's synchronisation stalls the pipeline, or processes whose device
// memory is fully reserved up front.  This entry point instead uses one
// file-scope device array of fixed size for that scratch; the caller passes
// device-resident queries and outputs, and the index must already be loaded.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the status words that must start at zero are cleared on the
// stream at the start of every call.  Two calls whose GPU work overlaps (on
// different streams, or from different threads on one index) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "../../include/pilot.h"
#include "kernels.h"

namespace pilot {
IndexView index_view(pilot_index* ix);
int set_error(int status, const char* msg);
}  // namespace pilot

using namespace pilot;

namespace {

// The scratch: PILOT_NOALLOC_SCRATCH_BYTES per device, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PILOT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

pilot_status error(pilot_status s, const char* fmt, long long a = 0, long long b = 0, long long c = 0) {
    char buf[400];
    snprintf(buf, sizeof buf, fmt, a, b, c);
    return pilot_status(set_error(int(s), buf));
}

pilot_status cuda_error(cudaError_t e, const char* what) {
    cudaGetLastError();
    char buf[300];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return pilot_status(set_error(int(PILOT_ECUDA), buf));
}

// Device address of the scratch array on the current device, looked up once
// per device.  In host code g_noalloc_scratch names a host-side stand-in, not
// device memory, so kernels must be given this address instead.
pilot_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return error(PILOT_EINVAL, "device %lld out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return PILOT_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" pilot_status pilot_search_noalloc(pilot_index* index, const float* queries, int64_t nq, int k, int ef,
                                             int32_t* out_ids, float* out_dists, void* stream) {
    if (!index) return error(PILOT_EINVAL, "index is NULL");
    if (nq < 0) return error(PILOT_EINVAL, "nq = %lld < 0", nq);
    if (k < 1 || ef < k || ef > PILOT_MAX_EF)
        return error(PILOT_EINVAL, "need 1 <= k <= ef <= %lld (k = %lld, ef = %lld)", PILOT_MAX_EF, k, ef);
    if (nq == 0) return PILOT_OK;
    if (!queries || !out_ids || !out_dists) return error(PILOT_EINVAL, "NULL query or output buffer");
    const IndexView v = index_view(index);
    std::lock_guard<std::mutex> lock(*static_cast<std::mutex*>(v.mutex));
    cudaError_t e = cudaSetDevice(v.device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    if (!on_device(queries) || !on_device(out_ids) || !on_device(out_dists))
        return error(PILOT_EINVAL, "pilot_search_noalloc needs device-resident queries and outputs");
    const DevIndex& X = *v.dev;

    // the same defaults as pilot_search
    const SearchConfig cfg = default_search_config(X, k, ef);

    // scratch layout inside the static array
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_status = take(8 * 4);
    const size_t o_qpad = take(size_t(nq) * X.d_pad * 4);
    const size_t o_qp = take(size_t(nq) * X.qp_pad * 4);
    const size_t o_pos = take(size_t(nq) * cfg.fes_T * 4);
    const size_t o_qpb = take(size_t((nq + 127) / 128 * 128) * X.qp_pad * 2);
    const size_t o_lb = take(size_t(nq) * 8);
    const size_t o_bad = take(size_t(nq) * 4);
    if (off > PILOT_NOALLOC_SCRATCH_BYTES) {
        const size_t per_q = size_t(X.d_pad) * 4 + size_t(X.qp_pad) * 6 + size_t(cfg.fes_T) * 4 + 8 + 4;
        char buf[400];
        snprintf(buf, sizeof buf,
                 "nq = %lld needs %zu bytes of scratch but pilot_search_noalloc holds %zu bytes (about %zu queries "
                 "for this index); split the batch",
                 (long long)nq, off, size_t(PILOT_NOALLOC_SCRATCH_BYTES),
                 (size_t(PILOT_NOALLOC_SCRATCH_BYTES) - 2048) / per_q);
        return pilot_status(set_error(int(PILOT_EINVAL), buf));
    }
    unsigned char* base = nullptr;
    pilot_status ps = scratch_address(v.device, &base);
    if (ps != PILOT_OK) return ps;

    SearchIO io{};
    io.nq = nq;
    io.queries = queries;
    io.status = reinterpret_cast<int32_t*>(base + o_status);
    io.q_pad = reinterpret_cast<float*>(base + o_qpad);
    io.qp = reinterpret_cast<float*>(base + o_qp);
    io.fes_pos = reinterpret_cast<int32_t*>(base + o_pos);
    io.qp_bf16 = reinterpret_cast<uint16_t*>(base + o_qpb);
    io.fes_lb = reinterpret_cast<double*>(base + o_lb);
    io.bad_query = reinterpret_cast<int32_t*>(base + o_bad);
    io.out_ids = out_ids;
    io.out_dists = out_dists;
    io.counters = nullptr;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemsetAsync(io.status, 0, 8 * 4, st)) != cudaSuccess) return cuda_error(e, "clear status");
    if ((e = launch_project(X, io, st)) != cudaSuccess) return cuda_error(e, "projection kernel");
    if ((e = launch_fes_mma(X, io, st)) != cudaSuccess) return cuda_error(e, "FES tensor-core kernel");
    e = launch_search(X, cfg, io, st, v.num_sms);
    if (e == cudaErrorInvalidConfiguration) {
        cudaGetLastError();
        return error(PILOT_EINVAL, "shared memory for ef = %lld exceeds the device limit", ef);
    }
    if (e != cudaSuccess) return cuda_error(e, "search kernel");
    if ((e = cudaMemcpyAsync(v.status_host, io.status, 8 * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e, "read status");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    if (v.status_host[2]) return error(PILOT_ETIMEOUT, "%lld search warps gave up waiting for a row gather", v.status_host[2]);
    if (v.status_host[5]) return error(PILOT_ETIMEOUT, "%lld FES blocks gave up waiting for the tensor cores", v.status_host[5]);
    if (v.status_host[4]) return error(PILOT_ECUDA, "%lld queries hit the expansion cap", v.status_host[4]);
    if (v.status_host[6])
        return error(PILOT_ECUDA, "%lld out-of-range graph indices were skipped (checked build)", v.status_host[6]);
    if (v.status_host[0])
        return error(PILOT_EINVAL, "%lld queries hold NaN or infinity (their results are -1 / +inf)",
                     v.status_host[0]);
    return PILOT_OK;
}
