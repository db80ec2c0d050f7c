// project.cu -- query projection q' = q V[:, :d'] (Sec. 4.1 (1)).
//
// One warp per query.  The query row is checked for NaN / infinity, copied
// zero-padded into the search layout, and each projected component is the
// FP32 rounding of the exact dot product with the FP64 basis column, which is
// held as an exact-enough FP32 pair (hi, lo): sum_j q_j (hi_j + lo_j) is
// accumulated with TwoProduct / TwoSum (device_common.cuh).
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "kernels.h"

namespace pilot {
namespace {

constexpr int kWarps = 8;

__global__ void __launch_bounds__(kWarps * 32) project_kernel(DevIndex ix, SearchIO io) {
    extern __shared__ __align__(16) float sq_all[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* sq = sq_all + warp * ix.d_pad;
    const int64_t stride = int64_t(gridDim.x) * kWarps;
    for (int64_t q = int64_t(blockIdx.x) * kWarps + warp; q < io.nq; q += stride) {
        const float* src = io.queries + q * ix.d;
        bool bad = false;
        for (int i = lane; i < ix.d_pad; i += 32) {
            float v = 0.0f;
            if (i < ix.d) {
                v = src[i];
                bad |= !isfinite(v);
            }
            sq[i] = v;
            io.q_pad[q * ix.d_pad + i] = v;
        }
        unsigned anybad = __ballot_sync(kFull, bad);
        if (lane == 0) {
            io.bad_query[q] = anybad ? 1 : 0;
            if (anybad) atomicAdd(&io.status[0], 1);
        }
        __syncwarp();
        for (int c = lane; c < ix.qp_pad; c += 32) {
            float r = 0.0f;
            if (c < ix.dp && !anybad) {
                DF acc{0.0f, 0.0f};
                for (int j = 0; j < ix.d; ++j) {
                    float2 v = __ldg(ix.basis + int64_t(j) * ix.qp_pad + c);
                    ip_acc2(acc, sq[j], v.x, v.y);
                }
                r = __fadd_rn(acc.hi, acc.lo);
            }
            io.qp[q * ix.qp_pad + c] = r;
            if (io.qp_bf16) io.qp_bf16[umma_kmajor_offset(q, c, 128, ix.qp_pad)] = __bfloat16_as_ushort(__float2bfloat16_rn(r));
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_project(const DevIndex& ix, const SearchIO& io, cudaStream_t st) {
    if (io.nq == 0) return cudaSuccess;
    size_t smem = size_t(kWarps) * ix.d_pad * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    // at most 16 resident blocks per SM; the grid-stride loop covers the rest
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int64_t blocks = (io.nq + kWarps - 1) / kWarps;
    if (blocks > int64_t(sms) * 16) blocks = int64_t(sms) * 16;
    project_kernel<<<unsigned(blocks), kWarps * 32, smem, st>>>(ix, io);
    return cudaGetLastError();
}

}  // namespace pilot
