// fes_scores.cu -- candidate generation for fast entry selection (Sec. 5).
//
// Dense FES (Table 2, "FES (1 block)") scores every projected query against
// every entry vector: s_e = ||e||^2 - 2 q'.e for squared L2 (the query norm
// is common to a row) or s_e = -q'.e for inner product.  This kernel keeps,
// per query, the T best scores and a certified lower bound
//     LB = ||q'||^2 + s_(T+1) - Delta
// on the exact distance of every entry it did not keep, where s_(T+1) is the
// smallest score left out and Delta bounds the scoring error.  The search
// kernel then computes the exact FP32 distances of the T survivors, and only
// if the best of them is not certified below LB scans all entries exactly.
//
// Scores here are FP32 on the CUDA cores: one thread per query, entry tiles
// staged in shared memory.
#include <cfloat>

#include "device_common.cuh"
#include "kernels.h"

namespace pilot {
namespace {

constexpr int kT = 8;          // survivors per query
constexpr int kThreads = 128;  // queries per block
constexpr int kTile = 32;      // entries per shared-memory tile

template <int QP>
__global__ void __launch_bounds__(kThreads) fes_score_kernel(DevIndex ix, SearchIO io) {
    __shared__ __align__(16) float se[kTile * QP];
    __shared__ float sn[kTile];
    const int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const bool active = q < io.nq;
    float qv[QP];
    double qq = 0.0;
#pragma unroll
    for (int i = 0; i < QP; ++i) {
        qv[i] = active ? io.qp[q * ix.qp_pad + i] : 0.0f;
        qq += double(qv[i]) * double(qv[i]);
    }
    float best_s[kT + 1];
    int best_p[kT + 1];
#pragma unroll
    for (int i = 0; i <= kT; ++i) {
        best_s[i] = FLT_MAX;
        best_p[i] = -1;
    }
    for (int64_t t0 = 0; t0 < ix.n_entry; t0 += kTile) {
        __syncthreads();
        for (int i = threadIdx.x; i < kTile * QP; i += kThreads) {
            int64_t e = t0 + i / QP;
            se[i] = e < ix.n_entry ? ix.entry_f32[e * ix.qp_pad + (i % QP)] : 0.0f;
        }
        for (int i = threadIdx.x; i < kTile; i += kThreads)
            sn[i] = (t0 + i < ix.n_entry) ? ix.entry_norm2[t0 + i] : 0.0f;
        __syncthreads();
        const int m = ix.n_entry - t0 < kTile ? int(ix.n_entry - t0) : kTile;
        for (int j = 0; j < m; ++j) {
            float dot = 0.0f;
#pragma unroll
            for (int i = 0; i < QP; ++i) dot = fmaf(qv[i], se[j * QP + i], dot);
            float s = ix.metric == 0 ? (sn[j] - 2.0f * dot) : -dot;
            if (s < best_s[kT]) {
                best_s[kT] = s;
                best_p[kT] = int(t0 + j);
#pragma unroll
                for (int i = kT; i > 0; --i) {
                    if (best_s[i] < best_s[i - 1]) {
                        float ts = best_s[i];
                        best_s[i] = best_s[i - 1];
                        best_s[i - 1] = ts;
                        int tp = best_p[i];
                        best_p[i] = best_p[i - 1];
                        best_p[i - 1] = tp;
                    }
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int i = 0; i < kT; ++i) io.fes_pos[q * kT + i] = best_p[i];
    double lb = INFINITY;
    if (ix.n_entry > kT) {
        // |s_hat - s| <= 2^-23 emax^2 + (2 dp + 2) 2^-24 |q| emax; Delta doubles it.
        double qn = sqrt(qq), em = double(ix.entry_max_norm);
        double delta = ldexp(1.0, -22) * (em * em + double(ix.dp + 2) * qn * em) + 1e-300;
        lb = (ix.metric == 0 ? qq : 0.0) + double(best_s[kT]) - delta;
    }
    io.fes_lb[q] = lb;
}

}  // namespace

cudaError_t launch_fes_scores(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st) {
    if (io.nq == 0) return cudaSuccess;
    if (cfg.fes_T != kT) return cudaErrorInvalidValue;
    unsigned blocks = unsigned((io.nq + kThreads - 1) / kThreads);
    switch (ix.qp_pad) {
        case 64: fes_score_kernel<64><<<blocks, kThreads, 0, st>>>(ix, io); break;
        case 128: fes_score_kernel<128><<<blocks, kThreads, 0, st>>>(ix, io); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pilot
