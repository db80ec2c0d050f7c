// fes_mma.cu -- fast entry selection candidates on the 5th-generation tensor
// cores (Sec. 5, dense form of Table 2).
//
// Scores every projected query against every entry vector as one BF16 GEMM
// with FP32 accumulation, S = Qb Eb^T, and keeps per query the T best scores
// s_e = ||e||^2 - 2 S[q, e] (squared L2; the query norm is common to a row)
// or s_e = -S[q, e] (inner product) together with a certified lower bound
//     LB = ||q'||^2 + s_(T+1) - Delta
// on the exact distance of every entry left out; Delta bounds the BF16
// rounding of both operands, the accumulation and the final subtraction.
// The search kernel computes the survivors' exact distances and scans all
// entries exactly when its best survivor is not certified below LB.
//
// One CTA per 128 queries; 6 warps:
//   warp 0  one lane issues bulk copies: the query tile once, then entry tiles
//           of 256 rows through a ring of shared-memory stages;
//   warp 1  allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and
//           one lane issues tcgen05.mma (M = 128, N = 256, K = 16 per
//           instruction) for each entry tile, committing to barriers that
//           free the stage and hand the accumulator to the epilogue;
//   warps 2-9 the epilogue: two warps per 32-lane TMEM quarter, each taking
//           half of a tile's columns; a thread owns one query row, reads 32
//           columns at a time with tcgen05.ld, forms the scores and keeps a
//           sorted top-(T+1) in registers with a branchless insertion network
//           applied only to scores that some row of the warp needs; the two
//           halves' lists are merged at the end.
// Operands are stored in global memory already in the UMMA canonical K-major
// layout without swizzle (8 x 16-byte core matrices; K-adjacent core matrices
// 128 bytes apart, 8-row groups KP * 16 bytes apart), so each tile is one
// contiguous bulk copy.  Every barrier wait is bounded; on a timeout the CTA
// reports, finishes its loops and still frees its TMEM.
#include <cfloat>
#include <cstdint>

#include "device_common.cuh"
#include "kernels.h"

namespace pilot {
namespace {

constexpr int kM = 128;          // queries per CTA (MMA M)
constexpr int kN = 256;          // entries per tile (MMA N)
constexpr int kT = kFesT;        // survivors per query
constexpr uint32_t kPolls = 1u << 24;

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int kp) {
    // start address, leading (K) byte offset 128, stride (8-row) byte offset
    // kp * 16, descriptor version 1, no swizzle
    uint64_t d = 0;
    d |= uint64_t((saddr >> 4) & 0x3FFFu);
    d |= uint64_t(128u >> 4) << 16;
    d |= uint64_t((uint32_t(kp) * 16u >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kN >> 3) << 17) |
                            (uint32_t(kM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);

// Insert (v, p) into the ascending list s[0..kT] (dropping the largest),
// branch-free.
__device__ __forceinline__ void insert_sorted(float (&s)[kT + 1], int (&ps)[kT + 1], float v, int p) {
#pragma unroll
    for (int t = 0; t <= kT; ++t) {
        const bool sw = v < s[t];
        const float tv = sw ? s[t] : v;
        const int tp = sw ? ps[t] : p;
        s[t] = sw ? v : s[t];
        ps[t] = sw ? p : ps[t];
        v = tv;
        p = tp;
    }
}

struct Smem {
    uint64_t a_full, b_full[4], b_empty[4], t_full[2], t_empty[2];
    uint32_t tmem_base;
    int failed;
};

__global__ void __launch_bounds__(kThreads, 1) fes_mma_kernel(DevIndex ix, SearchIO io, int kp, int nstage) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Smem* sm = reinterpret_cast<Smem*>(base);
    uint8_t* a_tile = base + 1024;
    const int a_bytes = kM * kp * 2;
    const int b_bytes = kN * kp * 2;
    uint8_t* b_tiles = a_tile + a_bytes;
    // second-half lists for the final merge: kM rows x (kT + 1) (score, position)
    float* merge_s = reinterpret_cast<float*>(b_tiles + nstage * b_bytes);
    int* merge_p = reinterpret_cast<int*>(merge_s + kM * (kT + 1));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q0 = int64_t(blockIdx.x) * kM;
    const int n_tiles = int((ix.n_entry + kN - 1) / kN);

    if (threadIdx.x == 0) {
        mbar_init(&sm->a_full, 1);
        for (int s = 0; s < nstage; ++s) {
            mbar_init(&sm->b_full[s], 1);
            mbar_init(&sm->b_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sm->t_full[b], 1);
            mbar_init(&sm->t_empty[b], kEpiWarps);
        }
        sm->failed = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sm->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(&sm->a_full, uint32_t(a_bytes));
            bulk_copy_g2s(a_tile, io.qp_bf16 + q0 * kp, uint32_t(a_bytes), &sm->a_full);
            for (int j = 0; j < n_tiles; ++j) {
                const int s = j % nstage;
                if (!mbar_wait(&sm->b_empty[s], uint32_t(((j / nstage) + 1) & 1), kPolls)) {
                    sm->failed = 1;
                    break;
                }
                mbar_arrive_expect_tx(&sm->b_full[s], uint32_t(b_bytes));
                bulk_copy_g2s(b_tiles + s * b_bytes, ix.entry_bf16 + int64_t(j) * kN * kp, uint32_t(b_bytes),
                              &sm->b_full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(&sm->a_full, 0, kPolls);
            const uint32_t a_addr = smem_u32(a_tile);
            for (int j = 0; ok && j < n_tiles; ++j) {
                const int s = j % nstage, b = j & 1;
                if (!mbar_wait(&sm->b_full[s], uint32_t((j / nstage) & 1), kPolls) ||
                    !mbar_wait(&sm->t_empty[b], uint32_t(((j >> 1) + 1) & 1), kPolls)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t b_addr = smem_u32(b_tiles + s * b_bytes);
                for (int ks = 0; ks < kp / 16; ++ks)
                    mma_bf16(tmem + uint32_t(b * kN), smem_desc(a_addr + uint32_t(ks) * 256u, kp),
                             smem_desc(b_addr + uint32_t(ks) * 256u, kp), ks > 0 ? 1u : 0u);
                mma_commit(&sm->b_empty[s]);
                mma_commit(&sm->t_full[b]);
            }
            if (!ok) sm->failed = 1;
        }
    }
    // epilogue: warp w reads TMEM lanes 32 * (w % 4) .. + 31, columns of half h
    const bool epi = warp >= 2;
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const int64_t q = q0 + row;
    const bool active = q < io.nq;
    float best_s[kT + 1];
    int best_p[kT + 1];
#pragma unroll
    for (int i = 0; i <= kT; ++i) {
        best_s[i] = FLT_MAX;
        best_p[i] = -1;
    }
    if (epi) {
        for (int j = 0; j < n_tiles; ++j) {
            const int b = j & 1;
            if (!mbar_wait(&sm->t_full[b], uint32_t((j >> 1) & 1), kPolls)) {
                sm->failed = 1;
                break;
            }
            tc_fence_after();
            for (int c0 = half * (kN / 2); c0 < (half + 1) * (kN / 2); c0 += 32) {
                float v[32];
                tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * kN + c0), v);
                const int e0 = j * kN + c0;
                float sc[32];
                if (ix.metric == 0) {   // norms are padded with +inf past n_entry
                    const float4* nrm = reinterpret_cast<const float4*>(ix.entry_norm2 + e0);
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const float4 f = __ldg(nrm + t);
                        sc[4 * t + 0] = f.x - 2.0f * v[4 * t + 0];
                        sc[4 * t + 1] = f.y - 2.0f * v[4 * t + 1];
                        sc[4 * t + 2] = f.z - 2.0f * v[4 * t + 2];
                        sc[4 * t + 3] = f.w - 2.0f * v[4 * t + 3];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) sc[i] = e0 + i < ix.n_entry ? -v[i] : INFINITY;
                }
                float mn = sc[0];
#pragma unroll
                for (int i = 1; i < 32; ++i) mn = fminf(mn, sc[i]);
                // most chunks hold no score below any row's current (T+1)-th best
                if (__any_sync(kFull, mn < best_s[kT])) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (__any_sync(kFull, sc[i] < best_s[kT])) insert_sorted(best_s, best_p, sc[i], e0 + i);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&sm->t_empty[b]))
                                        : "memory");
        }
        if (half == 1) {
#pragma unroll
            for (int i = 0; i <= kT; ++i) {
                merge_s[row * (kT + 1) + i] = best_s[i];
                merge_p[row * (kT + 1) + i] = best_p[i];
            }
        }
    }
    __syncthreads();
    if (epi && half == 0) {
#pragma unroll 1
        for (int i = 0; i <= kT; ++i) insert_sorted(best_s, best_p, merge_s[row * (kT + 1) + i], merge_p[row * (kT + 1) + i]);
        if (active) {
            double qq = 0.0;
            for (int i = 0; i < kp; ++i) {
                const double v = double(io.qp[q * ix.qp_pad + i]);
                qq += v * v;
            }
#pragma unroll
            for (int i = 0; i < kT; ++i) io.fes_pos[q * kT + i] = best_p[i];
            double lb = INFINITY;
            if (ix.n_entry > kT) {
                // BF16 operands (relative 2^-9 each), FP32 accumulation of kp
                // products, the norm and the final subtraction, doubled
                const double qn = sqrt(qq), em = double(ix.entry_max_norm);
                const double delta = (ldexp(1.0, -7) + ldexp(1.0, -15) + double(kp) * ldexp(1.0, -19)) * qn * em +
                                     ldexp(1.0, -21) * (em * em + qn * em) + 1e-300;
                lb = (ix.metric == 0 ? qq : 0.0) + double(best_s[kT]) - delta;
            }
            io.fes_lb[q] = lb;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    if (threadIdx.x == 0 && sm->failed) atomicAdd(&io.status[5], 1);
}

}  // namespace

size_t fes_mma_smem(int kp, int nstage) {
    return 1024 + 1024 + size_t(kM) * kp * 2 + size_t(nstage) * kN * kp * 2 + size_t(kM) * (kT + 1) * 8;
}

int fes_mma_stages(int kp) { return kp <= 64 ? 4 : 2; }

cudaError_t launch_fes_mma(const DevIndex& ix, const SearchIO& io, cudaStream_t st) {
    if (io.nq == 0) return cudaSuccess;
    const int kp = ix.qp_pad;
    if (kp != 64 && kp != 128) return cudaErrorInvalidValue;
    const int nstage = fes_mma_stages(kp);
    const size_t smem = fes_mma_smem(kp, nstage);
    cudaError_t e = cudaFuncSetAttribute(fes_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    const unsigned blocks = unsigned((io.nq + kM - 1) / kM);
    fes_mma_kernel<<<blocks, kThreads, smem, st>>>(ix, io, kp, nstage);
    return cudaGetLastError();
}

}  // namespace pilot
