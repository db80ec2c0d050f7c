// pilot_api.cu -- the C ABI (include/pilot.h): index loading and validation,
// per-call workspace, and the launch sequence of a search.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/pilot.h"
#include "kernels.h"

using namespace pilot;

namespace {

thread_local std::string g_error;

pilot_status fail(pilot_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t e__ = (expr);                                                                   \
        if (e__ != cudaSuccess)                                                                     \
            return cudaGetLastError(), fail(e__ == cudaErrorMemoryAllocation ? PILOT_ENOMEM : PILOT_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e__), __FILE__, __LINE__);                        \
    } while (0)

int round_up(int x, int m) { return (x + m - 1) / m * m; }

double decode_e4m3_host(uint8_t c) {
    int e = (c >> 3) & 0xF, m = c & 7;
    double v = e == 0 ? std::ldexp(double(m), -9) : std::ldexp(1.0 + m / 8.0, e - 7);
    return (c & 0x80) ? -v : v;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Non-finite values among n floats in device memory (load-time validation of
// full vectors given as a device pointer).
__global__ void count_nonfinite_kernel(const float* p, int64_t n, unsigned long long* out) {
    unsigned long long c = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        c += !isfinite(p[i]);
    if (c) atomicAdd(out, c);
}

double decode_bf16_host(uint16_t h) {
    uint32_t b = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

}  // namespace

struct pilot_index {
    DevIndex dev{};
    std::vector<void*> allocs;
    int device = 0;
    int num_sms = 0;
    std::mutex mu;
    // per-call workspace (grow-only)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int32_t* status_host = nullptr;   // pinned
    size_t device_bytes = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};   // per-kernel timing (on request)
    TunedShape tuned[kEfClasses] = {};   // autotuned search shapes by ef class

    std::vector<void*> host_allocs;   // pinned, mapped (host-resident full vectors)

    ~pilot_index() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (void* p : allocs) cudaFree(p);
        for (void* p : host_allocs) cudaFreeHost(p);
        if (ws) cudaFree(ws);
        if (status_host) cudaFreeHost(status_host);
    }

    template <class T>
    pilot_status upload(const T* host, size_t count, const T** out) {
        void* p = nullptr;
        size_t bytes = std::max<size_t>(count * sizeof(T), 16);
        CUDA_TRY(cudaMalloc(&p, bytes));
        allocs.push_back(p);
        device_bytes += bytes;
        if (count) CUDA_TRY(cudaMemcpy(p, host, count * sizeof(T), cudaMemcpyHostToDevice));
        *out = static_cast<const T*>(p);
        return PILOT_OK;
    }

    // rows x width elements of esize bytes into rows x pitch_bytes, zero padded
    // Rows copied into pinned host memory mapped into the device's address
    // space; *out is the device-side address.
    pilot_status map_rows(const void* src, int64_t rows, size_t width_bytes, size_t pitch_bytes, bool src_dev,
                          const void** out) {
        void* h = nullptr;
        size_t bytes = std::max<size_t>(size_t(rows) * pitch_bytes, 16);
        CUDA_TRY(cudaHostAlloc(&h, bytes, cudaHostAllocMapped));
        host_allocs.push_back(h);
        if (pitch_bytes != width_bytes) std::memset(h, 0, bytes);
        if (src_dev) {   // straight from device memory into the pinned rows
            if (rows)
                CUDA_TRY(cudaMemcpy2D(h, pitch_bytes, src, width_bytes, width_bytes, size_t(rows),
                                      cudaMemcpyDeviceToHost));
        } else {
            for (int64_t r = 0; r < rows; ++r)
                std::memcpy(static_cast<char*>(h) + size_t(r) * pitch_bytes,
                            static_cast<const char*>(src) + size_t(r) * width_bytes, width_bytes);
        }
        void* d = nullptr;
        CUDA_TRY(cudaHostGetDevicePointer(&d, h, 0));
        *out = d;
        return PILOT_OK;
    }

    pilot_status upload_rows(const void* host, int64_t rows, size_t width_bytes, size_t pitch_bytes,
                             const void** out) {
        void* p = nullptr;
        size_t bytes = std::max<size_t>(size_t(rows) * pitch_bytes, 16);
        CUDA_TRY(cudaMalloc(&p, bytes));
        allocs.push_back(p);
        device_bytes += bytes;
        if (pitch_bytes != width_bytes) CUDA_TRY(cudaMemset(p, 0, bytes));
        if (rows)
            CUDA_TRY(cudaMemcpy2D(p, pitch_bytes, host, width_bytes, width_bytes, size_t(rows), cudaMemcpyDefault));
        *out = p;
        return PILOT_OK;
    }
};

namespace pilot {

// Internal helpers for entry points defined in other translation units.
IndexView index_view(pilot_index* ix) {
    return IndexView{&ix->dev, ix->device, ix->num_sms, ix->status_host, &ix->mu, ix->tuned};
}

int set_error(int status, const char* msg) {
    g_error = msg;
    return status;
}

}  // namespace pilot

extern "C" {

const char* pilot_last_error(void) { return g_error.c_str(); }

int pilot_abi_version(void) { return 5; }

void pilot_search_options_default(pilot_search_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->stage1 = 1;
    opt->stage2_expansions = 2;
    opt->stage3 = 1;
    opt->use_fes = 1;
    opt->fes_seeds = 1;
}

void pilot_index_free(pilot_index* index) { delete index; }

pilot_status pilot_index_info(const pilot_index* index, int64_t* n, int64_t* d, int64_t* dp, int64_t* n_sub,
                              int64_t* device_bytes) {
    if (!index) return fail(PILOT_EINVAL, "index is NULL");
    if (n) *n = index->dev.n;
    if (d) *d = index->dev.d;
    if (dp) *dp = index->dev.dp;
    if (n_sub) *n_sub = index->dev.n_sub;
    if (device_bytes) *device_bytes = int64_t(index->device_bytes);
    return PILOT_OK;
}

static pilot_status validate_rows(const int32_t* adj, int64_t rows, int64_t width, int64_t n, const uint8_t* mask,
                                  bool sub, const char* what) {
    std::vector<int64_t> stamp(size_t(n), -1);
    for (int64_t r = 0; r < rows; ++r) {
        const int32_t* row = adj + r * width;
        for (int64_t j = 0; j < width; ++j) {
            int32_t v = row[j];
            if (v < -1 || v >= n) return fail(PILOT_EINVAL, "%s row %lld holds id %d outside [-1, n)", what,
                                              (long long)r, v);
            if (v < 0) continue;
            if (sub && !mask[r]) return fail(PILOT_EINVAL, "%s row %lld of an unsampled node is not empty", what,
                                             (long long)r);
            if (sub && !mask[v]) return fail(PILOT_EINVAL, "%s edge %lld -> %d reaches an unsampled node", what,
                                             (long long)r, v);
            if (stamp[v] == r) return fail(PILOT_EINVAL, "%s row %lld repeats id %d", what, (long long)r, v);
            stamp[v] = r;
        }
    }
    return PILOT_OK;
}

pilot_status pilot_index_load(const pilot_index_desc* dsc, pilot_index** out) {
    if (!dsc || !out) return fail(PILOT_EINVAL, "desc and out must not be NULL");
    *out = nullptr;
    const pilot_index_desc& D = *dsc;
    if (D.n < 1 || D.n >= (int64_t(1) << 31)) return fail(PILOT_EINVAL, "n = %lld out of range", (long long)D.n);
    if (D.d < 1 || D.d > 4096) return fail(PILOT_EINVAL, "d = %lld out of range [1, 4096]", (long long)D.d);
    if (D.dp < 1 || D.dp > D.d || D.dp > 128)
        return fail(PILOT_EINVAL, "dp = %lld must be in [1, min(d, 128)]", (long long)D.dp);
    if (D.R < 1 || D.R > PILOT_MAX_DEGREE || D.R_sub < 1 || D.R_sub > PILOT_MAX_DEGREE)
        return fail(PILOT_EINVAL, "R and R_sub must be in [1, %d]", PILOT_MAX_DEGREE);
    if (D.n_entry < 1) return fail(PILOT_EINVAL, "n_entry must be >= 1");
    if (D.full_vecs_location != PILOT_FULL_VECS_DEVICE && D.full_vecs_location != PILOT_FULL_VECS_HOST)
        return fail(PILOT_EINVAL, "full_vecs_location must be PILOT_FULL_VECS_DEVICE or PILOT_FULL_VECS_HOST");
    if (D.metric != PILOT_METRIC_L2 && D.metric != PILOT_METRIC_IP) return fail(PILOT_EINVAL, "bad metric");
    if (D.n_clusters < 0 || D.n_clusters > D.n_entry)
        return fail(PILOT_EINVAL, "n_clusters must be in [0, n_entry]");
    if (D.n_clusters > 0) {
        if (!D.entry_cluster || !D.cluster_centroids)
            return fail(PILOT_EINVAL, "entry_cluster and cluster_centroids are required when n_clusters > 0");
        std::vector<int64_t> size(size_t(D.n_clusters), 0);
        for (int64_t e = 0; e < D.n_entry; ++e) {
            if (D.entry_cluster[e] < 0 || D.entry_cluster[e] >= D.n_clusters)
                return fail(PILOT_EINVAL, "entry_cluster[%lld] out of range", (long long)e);
            size[size_t(D.entry_cluster[e])] += 1;
        }
        for (int64_t c = 0; c < D.n_clusters; ++c)
            if (size[size_t(c)] == 0) return fail(PILOT_EINVAL, "cluster %lld has no entry", (long long)c);
        for (int64_t i = 0; i < D.n_clusters * D.dp; ++i)
            if (!std::isfinite(D.cluster_centroids[i])) return fail(PILOT_EINVAL, "a centroid is not finite");
    }
    if (D.reduced_dtype < 0 || D.reduced_dtype > 2) return fail(PILOT_EINVAL, "bad reduced_dtype");
    if (!D.graph || !D.subgraph_mask || !D.subgraph || !D.svd_basis || !D.reduced_vecs || !D.full_vecs ||
        !D.entry_ids)
        return fail(PILOT_EINVAL, "a required array is NULL");
    if ((D.reduced_dtype == PILOT_REDUCED_FP8_E4M3) != (D.reduced_scales != nullptr))
        return fail(PILOT_EINVAL, "reduced_scales must be given exactly for FP8 rows");

    const int64_t n = D.n, d = D.d, dp = D.dp;
    std::vector<int32_t> sub2full, full2sub(size_t(n), -1);
    for (int64_t v = 0; v < n; ++v) {
        if (D.subgraph_mask[v] > 1) return fail(PILOT_EINVAL, "subgraph_mask must hold 0 or 1");
        if (D.subgraph_mask[v]) {
            full2sub[size_t(v)] = int32_t(sub2full.size());
            sub2full.push_back(int32_t(v));
        }
    }
    const int64_t n_sub = int64_t(sub2full.size());
    if (n_sub < 1) return fail(PILOT_EINVAL, "the subgraph samples no node");
    pilot_status s;
    if ((s = validate_rows(D.graph, n, D.R, n, nullptr, false, "graph")) != PILOT_OK) return s;
    if ((s = validate_rows(D.subgraph, n, D.R_sub, n, D.subgraph_mask, true, "subgraph")) != PILOT_OK) return s;
    for (int64_t e = 0; e < D.n_entry; ++e) {
        int32_t v = D.entry_ids[e];
        if (v < 0 || v >= n || !D.subgraph_mask[v])
            return fail(PILOT_EINVAL, "entry %lld (id %d) is not a sampled node", (long long)e, v);
    }
    // full vectors may be given in device memory (of the current device)
    const bool full_dev = is_device_ptr(D.full_vecs);
    if (full_dev) {
        unsigned long long* cnt = nullptr;
        unsigned long long bad = 0;
        int dev = 0, sms = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CUDA_TRY(cudaMalloc(&cnt, sizeof bad));
        cudaError_t e1 = cudaMemset(cnt, 0, sizeof bad);
        if (e1 == cudaSuccess) {
            count_nonfinite_kernel<<<unsigned(sms * 8), 256>>>(D.full_vecs, n * d, cnt);
            e1 = cudaGetLastError();
        }
        if (e1 == cudaSuccess) e1 = cudaMemcpy(&bad, cnt, sizeof bad, cudaMemcpyDeviceToHost);
        cudaFree(cnt);
        CUDA_TRY(e1);
        if (bad) return fail(PILOT_EINVAL, "full_vecs holds a non-finite value");
    } else {
        for (int64_t i = 0; i < n * d; ++i)
            if (!std::isfinite(D.full_vecs[i])) return fail(PILOT_EINVAL, "full_vecs holds a non-finite value");
    }
    for (int64_t i = 0; i < d * dp; ++i)
        if (!std::isfinite(D.svd_basis[i])) return fail(PILOT_EINVAL, "svd_basis holds a non-finite value");

    const int esize = D.reduced_dtype == 0 ? 4 : (D.reduced_dtype == 1 ? 2 : 1);
    auto red_value = [&](int64_t r, int64_t c) -> double {
        int64_t at = r * dp + c;
        if (D.reduced_dtype == 0) return double(static_cast<const float*>(D.reduced_vecs)[at]);
        if (D.reduced_dtype == 1) return decode_bf16_host(static_cast<const uint16_t*>(D.reduced_vecs)[at]);
        return decode_e4m3_host(static_cast<const uint8_t*>(D.reduced_vecs)[at]) * double(D.reduced_scales[r]);
    };
    if (D.reduced_dtype == 2) {
        const uint8_t* codes = static_cast<const uint8_t*>(D.reduced_vecs);
        for (int64_t i = 0; i < n_sub * dp; ++i)
            if ((codes[i] & 0x7F) == 0x7F) return fail(PILOT_EINVAL, "reduced_vecs holds an FP8 NaN code");
        for (int64_t r = 0; r < n_sub; ++r)
            if (!(D.reduced_scales[r] > 0.0f) || !std::isfinite(D.reduced_scales[r]))
                return fail(PILOT_EINVAL, "reduced_scales must be finite and > 0");
    } else {
        for (int64_t r = 0; r < n_sub; ++r)
            for (int64_t c = 0; c < dp; ++c)
                if (!std::isfinite(red_value(r, c))) return fail(PILOT_EINVAL, "reduced_vecs holds a non-finite value");
    }

    auto* ix = new pilot_index();
    std::unique_ptr<pilot_index> guard(ix);
    CUDA_TRY(cudaGetDevice(&ix->device));
    CUDA_TRY(cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, ix->device));
    DevIndex& X = ix->dev;
    X.n = n;
    X.d = d;
    X.dp = dp;
    X.n_sub = n_sub;
    X.n_entry = D.n_entry;
    X.R = int(D.R);
    X.R_sub = int(D.R_sub);
    X.metric = D.metric;
    X.red_dtype = D.reduced_dtype;
    X.d_pad = round_up(int(d), 32);
    X.full_row_bytes = X.d_pad * 4;
    X.red_row_bytes = round_up(int(dp) * esize, 128);
    X.dp_pad = X.red_row_bytes / esize;
    X.qp_pad = std::max(round_up(int(dp), 64), X.dp_pad);

    // compact subgraph (ids of sampled rows in ascending original order)
    std::vector<int32_t> sub_adj(size_t(n_sub * D.R_sub));
    for (int64_t c = 0; c < n_sub; ++c)
        for (int64_t j = 0; j < D.R_sub; ++j) {
            int32_t v = D.subgraph[int64_t(sub2full[c]) * D.R_sub + j];
            sub_adj[size_t(c * D.R_sub + j)] = v < 0 ? -1 : full2sub[size_t(v)];
        }
    // basis as (hi, lo) FP32 pairs, zero beyond dp
    std::vector<float2> basis(size_t(d * X.qp_pad), make_float2(0.f, 0.f));
    for (int64_t j = 0; j < d; ++j)
        for (int64_t c = 0; c < dp; ++c) {
            double v = D.svd_basis[j * dp + c];
            float hi = float(v);
            float lo = float(v - double(hi));
            basis[size_t(j * X.qp_pad + c)] = make_float2(hi, lo);
        }
    // entries: compact ids, decoded rows, norms
    std::vector<int32_t> entry(size_t(D.n_entry));
    std::vector<float> entry_f32(size_t(D.n_entry * X.qp_pad), 0.f), entry_n2(size_t(D.n_entry));
    double emax = 0.0;
    for (int64_t e = 0; e < D.n_entry; ++e) {
        int32_t c = full2sub[size_t(D.entry_ids[e])];
        entry[size_t(e)] = c;
        double nn = 0.0;
        for (int64_t k = 0; k < dp; ++k) {
            double v = red_value(c, k);
            entry_f32[size_t(e * X.qp_pad + k)] = float(v);
            nn += v * v;
        }
        entry_n2[size_t(e)] = float(nn);
        emax = std::max(emax, std::sqrt(nn));
    }
    X.entry_max_norm = float(emax * (1.0 + 1e-6));
    // BF16 copy for the tensor-core FES scores: RNE of the decoded values,
    // whole 256-row tiles (zero rows past n_entry) in the UMMA layout
    const int64_t e_tiles = (D.n_entry + 255) / 256;
    std::vector<uint16_t> entry_bf16(size_t(e_tiles * 256 * X.qp_pad), 0);
    for (int64_t e = 0; e < D.n_entry; ++e)
        for (int c = 0; c < X.qp_pad; ++c) {
            uint32_t b;
            std::memcpy(&b, &entry_f32[size_t(e * X.qp_pad + c)], 4);
            const uint32_t r = (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
            entry_bf16[size_t(umma_kmajor_offset(e, c, 256, X.qp_pad))] = uint16_t(r);
        }

    if ((s = ix->upload(D.graph, size_t(n * D.R), &X.graph)) != PILOT_OK) return s;
    if ((s = ix->upload(sub_adj.data(), sub_adj.size(), &X.sub_adj)) != PILOT_OK) return s;
    if ((s = ix->upload(sub2full.data(), sub2full.size(), &X.sub2full)) != PILOT_OK) return s;
    if ((s = ix->upload(full2sub.data(), full2sub.size(), &X.full2sub)) != PILOT_OK) return s;
    if ((s = ix->upload(basis.data(), basis.size(), &X.basis)) != PILOT_OK) return s;
    if ((s = ix->upload(entry.data(), entry.size(), &X.entry)) != PILOT_OK) return s;
    entry_n2.resize(size_t(e_tiles * 256), INFINITY);   // whole tiles; padded entries never score
    if ((s = ix->upload(entry_n2.data(), entry_n2.size(), &X.entry_norm2)) != PILOT_OK) return s;
    if ((s = ix->upload(entry_bf16.data(), entry_bf16.size(), &X.entry_bf16)) != PILOT_OK) return s;
    // clustered FES: FP32 centroid rows and the entries grouped by cluster
    X.n_clusters = int(D.n_clusters);
    X.cent_pad = round_up(int(dp), 32);
    if (D.n_clusters > 0) {
        std::vector<float> cent(size_t(D.n_clusters * X.cent_pad), 0.f);
        for (int64_t c = 0; c < D.n_clusters; ++c)
            for (int64_t k = 0; k < dp; ++k) cent[size_t(c * X.cent_pad + k)] = D.cluster_centroids[c * dp + k];
        std::vector<int32_t> off(size_t(D.n_clusters + 1), 0), grouped(size_t(D.n_entry));
        for (int64_t e = 0; e < D.n_entry; ++e) off[size_t(D.entry_cluster[e] + 1)] += 1;
        for (int64_t c = 0; c < D.n_clusters; ++c) off[size_t(c + 1)] += off[size_t(c)];
        std::vector<int32_t> fill(off.begin(), off.end() - 1);
        for (int64_t e = 0; e < D.n_entry; ++e) grouped[size_t(fill[size_t(D.entry_cluster[e])]++)] = entry[size_t(e)];
        if ((s = ix->upload(cent.data(), cent.size(), &X.centroids)) != PILOT_OK) return s;
        if ((s = ix->upload(grouped.data(), grouped.size(), &X.cl_entries)) != PILOT_OK) return s;
        if ((s = ix->upload(off.data(), off.size(), &X.cl_offsets)) != PILOT_OK) return s;
    }
    X.red_scales = nullptr;
    if (D.reduced_dtype == 2)
        if ((s = ix->upload(D.reduced_scales, size_t(n_sub), &X.red_scales)) != PILOT_OK) return s;
    const void* p = nullptr;
    if ((s = ix->upload_rows(D.reduced_vecs, n_sub, size_t(dp * esize), size_t(X.red_row_bytes), &p)) != PILOT_OK)
        return s;
    X.red = p;
    X.full_host = D.full_vecs_location == PILOT_FULL_VECS_HOST;
    if (X.full_host) {
        if ((s = ix->map_rows(D.full_vecs, n, size_t(d * 4), size_t(X.full_row_bytes), full_dev, &p)) != PILOT_OK)
            return s;
    } else if ((s = ix->upload_rows(D.full_vecs, n, size_t(d * 4), size_t(X.full_row_bytes), &p)) != PILOT_OK) {
        return s;
    }
    X.full = static_cast<const float*>(p);
    // visited sets: one hash table per warp slot the search kernel can keep
    // resident (16 per SM), each sized for the largest ef and the larger
    // degree -- independent of n above a small floor (64 KB per slot at
    // degree 32)
    {
        X.id_bits = 1;
        while ((int64_t(1) << X.id_bits) < n) ++X.id_bits;   // n - 1 < 2^id_bits <= 2^31
        X.epoch_max = kVisEpochs;
        // a shorter epoch cycle (more frequent table clears) for tests of the wrap
        if (const char* ev = std::getenv("PILOT_VISITED_EPOCH_CYCLE")) {
            const long long c = std::atoll(ev);
            if (c >= 1 && uint64_t(c) < X.epoch_max) X.epoch_max = uint32_t(c);
        }
        X.vis_stride = vis_entries_for(PILOT_MAX_EF, std::max(X.R, X.R_sub), X.id_bits);
        const int64_t slots = int64_t(ix->num_sms) * 16;
        X.vis_slots = int(slots);
        const size_t bytes = size_t(slots) * size_t(X.vis_stride) * sizeof(uint16_t);
        void* p1 = nullptr;
        CUDA_TRY(cudaMalloc(&p1, bytes));
        ix->allocs.push_back(p1);
        CUDA_TRY(cudaMemset(p1, 0, bytes));
        X.vis = static_cast<uint16_t*>(p1);
        void* p2 = nullptr;
        CUDA_TRY(cudaMalloc(&p2, size_t(slots) * 4));
        ix->allocs.push_back(p2);
        CUDA_TRY(cudaMemset(p2, 0, size_t(slots) * 4));
        X.vis_epoch = static_cast<uint32_t*>(p2);
        ix->device_bytes += bytes + size_t(slots) * 4;
    }
    CUDA_TRY(cudaMallocHost(&ix->status_host, 8 * sizeof(int32_t)));
    *out = guard.release();
    return PILOT_OK;
}


static uint64_t checksum64(const std::vector<char>& b) {
    uint64_t sum = 0;
    size_t nw = (b.size() + 7) / 8;
    for (size_t i = 0; i < nw; ++i) {
        uint64_t w = 0;
        size_t take = std::min<size_t>(8, b.size() - i * 8);
        std::memcpy(&w, b.data() + i * 8, take);   // little-endian host
        sum += w * (2 * uint64_t(i) + 1);
    }
    return sum;
}

pilot_status pilot_index_load_files(const char* dir, int flags, pilot_index** out) {
    if (!dir || !out) return fail(PILOT_EINVAL, "dir and out must not be NULL");
    if (flags & ~PILOT_LOAD_FULL_VECS_HOST) return fail(PILOT_EINVAL, "unknown flags %d", flags);
    *out = nullptr;
    const std::string root(dir);
    std::ifstream hdr(root + "/pilot_index.txt");
    if (!hdr) return fail(PILOT_EIO, "cannot open %s/pilot_index.txt", dir);
    std::string line;
    if (!std::getline(hdr, line) || line != "pilot-index 1") return fail(PILOT_EFORMAT, "bad header line");
    std::map<std::string, int64_t> meta;
    std::map<std::string, std::vector<char>> arrays;
    while (std::getline(hdr, line)) {
        if (line.empty()) continue;
        std::istringstream ls(line);
        std::string key;
        ls >> key;
        if (key == "array") {
            std::string name, kind, sum_hex;
            long long bytes = -1;
            ls >> name >> kind >> bytes >> sum_hex;
            if (!ls || bytes < 0) return fail(PILOT_EFORMAT, "bad array line: %s", line.c_str());
            std::ifstream f(root + "/" + name + ".bin", std::ios::binary | std::ios::ate);
            if (!f) return fail(PILOT_EIO, "cannot open %s.bin", name.c_str());
            if (int64_t(f.tellg()) != bytes) return fail(PILOT_EFORMAT, "%s.bin has the wrong size", name.c_str());
            f.seekg(0);
            std::vector<char> buf(static_cast<size_t>(bytes));
            if (bytes && !f.read(buf.data(), bytes)) return fail(PILOT_EIO, "cannot read %s.bin", name.c_str());
            if (checksum64(buf) != std::stoull(sum_hex, nullptr, 16))
                return fail(PILOT_EFORMAT, "%s.bin fails its checksum", name.c_str());
            arrays[name] = std::move(buf);
        } else {
            long long v;
            if (!(ls >> v)) return fail(PILOT_EFORMAT, "bad line: %s", line.c_str());
            meta[key] = v;
        }
    }
    for (const char* k : {"n", "d", "dp", "R", "R_sub", "n_sub", "n_entry", "metric", "reduced_dtype"})
        if (!meta.count(k)) return fail(PILOT_EFORMAT, "missing key %s", k);
    const int64_t n = meta["n"], d = meta["d"], dp = meta["dp"], R = meta["R"], Rs = meta["R_sub"];
    const int64_t ns = meta["n_sub"], ne = meta["n_entry"];
    const int dt = int(meta["reduced_dtype"]);
    const int es = dt == 0 ? 4 : (dt == 1 ? 2 : 1);
    struct Need { const char* name; int64_t bytes; };
    std::vector<Need> need = {{"graph", n * R * 4}, {"subgraph_mask", n}, {"subgraph", n * Rs * 4},
                              {"svd_basis", 0}, {"basis", d * dp * 8}, {"reduced", ns * dp * es},
                              {"full", n * d * 4}, {"entry_ids", ne * 4}};
    for (auto& nd : need) {
        if (nd.bytes == 0) continue;
        auto it = arrays.find(nd.name);
        if (it == arrays.end()) return fail(PILOT_EFORMAT, "missing array %s", nd.name);
        if (int64_t(it->second.size()) != nd.bytes) return fail(PILOT_EFORMAT, "array %s has the wrong size", nd.name);
    }
    if (dt == 2 && (!arrays.count("reduced_scales") || int64_t(arrays["reduced_scales"].size()) != ns * 4))
        return fail(PILOT_EFORMAT, "missing or short reduced_scales");
    const uint8_t* mask = reinterpret_cast<const uint8_t*>(arrays["subgraph_mask"].data());
    int64_t cnt = 0;
    for (int64_t v = 0; v < n; ++v) cnt += mask[v] != 0;
    if (cnt != ns) return fail(PILOT_EFORMAT, "n_sub does not match subgraph_mask");
    pilot_index_desc D{};
    D.n = n; D.d = d; D.dp = dp; D.R = R; D.R_sub = Rs; D.n_entry = ne;
    D.metric = int32_t(meta["metric"]);
    D.reduced_dtype = dt;
    D.graph = reinterpret_cast<const int32_t*>(arrays["graph"].data());
    D.subgraph_mask = mask;
    D.subgraph = reinterpret_cast<const int32_t*>(arrays["subgraph"].data());
    D.svd_basis = reinterpret_cast<const double*>(arrays["basis"].data());
    D.reduced_vecs = arrays["reduced"].data();
    D.reduced_scales = dt == 2 ? reinterpret_cast<const float*>(arrays["reduced_scales"].data()) : nullptr;
    D.full_vecs = reinterpret_cast<const float*>(arrays["full"].data());
    D.entry_ids = reinterpret_cast<const int32_t*>(arrays["entry_ids"].data());
    D.full_vecs_location = (flags & PILOT_LOAD_FULL_VECS_HOST) ? PILOT_FULL_VECS_HOST : PILOT_FULL_VECS_DEVICE;
    if (meta.count("n_clusters")) {   // optional entry clusters (clustered FES)
        const int64_t nc = meta["n_clusters"];
        if (!arrays.count("entry_cluster") || int64_t(arrays["entry_cluster"].size()) != ne * 4 ||
            !arrays.count("cluster_centroids") || int64_t(arrays["cluster_centroids"].size()) != nc * dp * 4)
            return fail(PILOT_EFORMAT, "missing or short entry_cluster / cluster_centroids");
        D.n_clusters = nc;
        D.entry_cluster = reinterpret_cast<const int32_t*>(arrays["entry_cluster"].data());
        D.cluster_centroids = reinterpret_cast<const float*>(arrays["cluster_centroids"].data());
    }
    return pilot_index_load(&D, out);
}


static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

pilot_status pilot_search_ex(pilot_index* ix, const float* queries, int64_t nq, int k, int ef, int32_t* out_ids,
                             float* out_dists, void* stream, const pilot_search_options* opt_in) {
    if (!ix) return fail(PILOT_EINVAL, "index is NULL");
    if (nq < 0) return fail(PILOT_EINVAL, "nq < 0");
    if (k < 1) return fail(PILOT_EINVAL, "k = %d < 1", k);
    if (ef < k) return fail(PILOT_EINVAL, "ef = %d < k = %d", ef, k);
    if (ef > PILOT_MAX_EF) return fail(PILOT_EINVAL, "ef = %d > %d", ef, PILOT_MAX_EF);
    if (nq > 0 && (!queries || !out_ids || !out_dists)) return fail(PILOT_EINVAL, "NULL query or output buffer");
    pilot_search_options opt;
    pilot_search_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.stage2_expansions < 0) return fail(PILOT_EINVAL, "stage2_expansions < 0");
    if (opt.fes_seeds == 0) opt.fes_seeds = 1;
    if (opt.fes_seeds < 1 || opt.fes_seeds > kFesT)
        return fail(PILOT_EINVAL, "fes_seeds = %d outside [1, %d]", opt.fes_seeds, kFesT);
    if (opt.seed_ids) {
        if (opt.stage1 || opt.stage2_expansions != 0 || !opt.stage3)
            return fail(PILOT_EINVAL, "seed_ids seed the final stage alone: stage1 = 0, stage2_expansions = 0, "
                                      "stage3 = 1");
        if (opt.seed_count < 1 || opt.seed_count > ef)
            return fail(PILOT_EINVAL, "seed_count = %d outside [1, ef = %d]", opt.seed_count, ef);
        if (is_device_ptr(opt.seed_ids)) return fail(PILOT_EINVAL, "seed_ids must be host memory");
        std::vector<int32_t> row(size_t(opt.seed_count));
        for (int64_t q = 0; q < nq; ++q) {
            const int32_t* r = opt.seed_ids + q * opt.seed_count;
            size_t n_ok = 0;
            for (int j = 0; j < opt.seed_count; ++j) {
                if (r[j] == -1) continue;
                if (r[j] < 0 || int64_t(r[j]) >= ix->dev.n)
                    return fail(PILOT_EINVAL, "seed id %d of query %lld out of range", r[j], (long long)q);
                row[n_ok++] = r[j];
            }
            std::sort(row.begin(), row.begin() + n_ok);
            if (std::adjacent_find(row.begin(), row.begin() + n_ok) != row.begin() + n_ok)
                return fail(PILOT_EINVAL, "seed ids of query %lld repeat", (long long)q);
        }
    }
    if (nq == 0) return PILOT_OK;
    std::lock_guard<std::mutex> lock(ix->mu);
    CUDA_TRY(cudaSetDevice(ix->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const DevIndex& X = ix->dev;

    SearchConfig cfg = default_search_config(X, k, ef);
    cfg.stage1 = opt.stage1 != 0;
    cfg.stage2_expansions = opt.stage2_expansions;
    cfg.stage3 = opt.stage3 != 0;
    if (opt.use_fes < 0 || opt.use_fes > 2) return fail(PILOT_EINVAL, "use_fes = %d outside [0, 2]", opt.use_fes);
    if (opt.use_fes == 2 && X.n_clusters < 1) return fail(PILOT_EINVAL, "use_fes = 2 needs an index with entry clusters");
    cfg.use_fes = opt.use_fes;
    cfg.fes_seeds = opt.fes_seeds;
    // explicit options first, then the autotuned shape of this ef class, then the defaults
    const TunedShape& tuned = ix->tuned[ef_class(ef)];
    const int wpb = opt.warps_per_block > 0 ? opt.warps_per_block : tuned.warps_per_block;
    const int rows = opt.stage_rows > 0 ? opt.stage_rows : tuned.stage_rows;
    if (wpb > 0) cfg.warps_per_block = std::min(wpb, 8);
    if (rows > 0) set_stage_rows(X, cfg, rows);
    if (opt.visited_entries != 0) {
        const int64_t v = opt.visited_entries;
        const int64_t vmin = vis_min_entries(X.id_bits);
        if (v < vmin || v > X.vis_stride || (v & (v - 1)))
            return fail(PILOT_EINVAL, "visited_entries = %lld must be 0 or a power of two in [%lld, %lld]",
                        (long long)v, (long long)vmin, (long long)X.vis_stride);
        set_visited_size(X, cfg, v);
    }

    const bool q_dev = is_device_ptr(queries);
    const bool ids_dev = is_device_ptr(out_ids), dists_dev = is_device_ptr(out_dists);
    const bool cnt_dev = opt.counters ? is_device_ptr(opt.counters) : true;

    // workspace layout
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
    const size_t o_q = q_dev ? 0 : take(size_t(nq) * X.d * 4);
    const size_t o_ids = ids_dev ? 0 : take(size_t(nq) * k * 4);
    const size_t o_dists = dists_dev ? 0 : take(size_t(nq) * k * 4);
    const size_t o_cnt = (opt.counters && !cnt_dev) ? take(size_t(nq) * 8 * 4) : 0;
    const size_t o_seed = opt.seed_ids ? take(size_t(nq) * opt.seed_count * 4) : 0;
    if (off > ix->ws_bytes) {
        if (ix->ws) cudaFree(ix->ws);
        ix->ws = nullptr;
        ix->ws_bytes = 0;
        CUDA_TRY(cudaMalloc(&ix->ws, off));
        ix->ws_bytes = off;
    }
    char* ws = static_cast<char*>(ix->ws);
    SearchIO io{};
    io.nq = nq;
    io.status = reinterpret_cast<int32_t*>(ws + o_status);
    io.q_pad = reinterpret_cast<float*>(ws + o_qpad);
    io.qp = reinterpret_cast<float*>(ws + o_qp);
    io.fes_pos = reinterpret_cast<int32_t*>(ws + o_pos);
    io.qp_bf16 = reinterpret_cast<uint16_t*>(ws + o_qpb);
    io.fes_lb = reinterpret_cast<double*>(ws + o_lb);
    io.bad_query = reinterpret_cast<int32_t*>(ws + o_bad);
    io.queries = q_dev ? queries : reinterpret_cast<const float*>(ws + o_q);
    io.out_ids = ids_dev ? out_ids : reinterpret_cast<int32_t*>(ws + o_ids);
    io.out_dists = dists_dev ? out_dists : reinterpret_cast<float*>(ws + o_dists);
    io.counters = opt.counters ? (cnt_dev ? opt.counters : reinterpret_cast<int32_t*>(ws + o_cnt)) : nullptr;
    io.seed_ids = opt.seed_ids ? reinterpret_cast<const int32_t*>(ws + o_seed) : nullptr;
    io.seed_count = opt.seed_ids ? opt.seed_count : 0;

    CUDA_TRY(cudaMemsetAsync(io.status, 0, 8 * 4, st));
    if (!q_dev)
        CUDA_TRY(cudaMemcpyAsync(const_cast<float*>(io.queries), queries, size_t(nq) * X.d * 4,
                                 cudaMemcpyHostToDevice, st));
    if (opt.seed_ids)
        CUDA_TRY(cudaMemcpyAsync(const_cast<int32_t*>(io.seed_ids), opt.seed_ids, size_t(nq) * opt.seed_count * 4,
                                 cudaMemcpyHostToDevice, st));
    const bool timed = opt.kernel_ms != nullptr;
    if (timed && !ix->ev[0])
        for (cudaEvent_t& e : ix->ev) CUDA_TRY(cudaEventCreate(&e));
    if (timed) CUDA_TRY(cudaEventRecord(ix->ev[0], st));
    CUDA_TRY(launch_project(X, io, st));
    if (timed) CUDA_TRY(cudaEventRecord(ix->ev[1], st));
    if (cfg.use_fes == 1 && !opt.seed_ids) CUDA_TRY(launch_fes_mma(X, io, st));
    if (timed) CUDA_TRY(cudaEventRecord(ix->ev[2], st));
    {
        cudaError_t e = launch_search(X, cfg, io, st, ix->num_sms);
        if (e == cudaErrorInvalidConfiguration) {
            cudaGetLastError();
            return fail(PILOT_EINVAL, "per-block shared memory (%zu B per warp x %d warps) exceeds the device limit; "
                        "lower ef or warps_per_block", search_smem_per_warp(X, cfg), cfg.warps_per_block);
        }
        CUDA_TRY(e);
    }
    if (timed) CUDA_TRY(cudaEventRecord(ix->ev[3], st));
    if (!ids_dev) CUDA_TRY(cudaMemcpyAsync(out_ids, io.out_ids, size_t(nq) * k * 4, cudaMemcpyDeviceToHost, st));
    if (!dists_dev)
        CUDA_TRY(cudaMemcpyAsync(out_dists, io.out_dists, size_t(nq) * k * 4, cudaMemcpyDeviceToHost, st));
    if (opt.counters && !cnt_dev)
        CUDA_TRY(cudaMemcpyAsync(opt.counters, io.counters, size_t(nq) * 8 * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(ix->status_host, io.status, 8 * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (timed)
        for (int i = 0; i < 3; ++i) CUDA_TRY(cudaEventElapsedTime(&opt.kernel_ms[i], ix->ev[i], ix->ev[i + 1]));
    const int32_t* S = ix->status_host;
    if (opt.status_words) std::memcpy(opt.status_words, S, 8 * sizeof(int32_t));
    if (S[2]) return fail(PILOT_ETIMEOUT, "%d search warps gave up waiting for a row gather", S[2]);
    if (S[5]) return fail(PILOT_ETIMEOUT, "%d FES blocks gave up waiting for the tensor cores", S[5]);
    if (S[4]) return fail(PILOT_ECUDA, "%d queries hit the expansion cap", S[4]);
    if (S[6]) return fail(PILOT_ECUDA, "%d out-of-range graph indices were skipped (checked build)", S[6]);
    if (S[0]) return fail(PILOT_EINVAL, "%d queries hold NaN or infinity (their results are -1 / +inf)", S[0]);
    return PILOT_OK;
}

pilot_status pilot_search(pilot_index* index, const float* queries, int64_t nq, int k, int ef, int32_t* out_ids,
                          float* out_dists, void* stream) {
    return pilot_search_ex(index, queries, nq, k, ef, out_ids, out_dists, stream, nullptr);
}

}  // extern "C"
