// device_common.cuh -- device helpers shared by the search kernels.
//
// Numerics.  The paper computes every distance in FP32 (Sec. 6.1).  Here each
// distance is the FP32 rounding of its exact value: the sum is carried as an
// unevaluated pair hi + lo of FP32 numbers built from error-free
// transformations -- Knuth's TwoSum and the FMA-based TwoProduct (as used in
// Ogita, Rump & Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 2005) -- and rounded once at the end.  The result is independent of the
// order in which lanes combine partial sums except in the rare case where the
// exact value lies within ~2^-40 (relative) of an FP32 rounding boundary.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

namespace pilot {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint64_t kKeyEmpty = ~0ull;

// ------------------------------------------------------------ FP32 pairs --

struct DF {
    float hi, lo;
};

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    float s = __fadd_rn(a, b);
    float bv = __fsub_rn(s, a);
    float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return s;
}

// p + e == a * b exactly (FMA).
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
    float p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
    return p;
}

// acc += (q - x)^2 with q - x = d + e exact, (d + e)^2 ~= d*d + 2de; d*d is
// split exactly, the small terms go to acc.lo.
__device__ __forceinline__ void l2_acc(DF& acc, float q, float x) {
    float e;
    float d = two_sum(q, -x, e);
    float pe;
    float p = two_prod(d, d, pe);
    float t;
    acc.hi = two_sum(acc.hi, p, t);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, __fmaf_rn(__fmul_rn(2.0f, d), e, pe)));
}

// Same with x = xh + xl given exactly as two FP32 numbers (FP8 code * scale).
__device__ __forceinline__ void l2_acc2(DF& acc, float q, float xh, float xl) {
    float e;
    float d = two_sum(q, -xh, e);
    e = __fsub_rn(e, xl);
    float pe;
    float p = two_prod(d, d, pe);
    float t;
    acc.hi = two_sum(acc.hi, p, t);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, __fmaf_rn(__fmul_rn(2.0f, d), e, pe)));
}

// acc += q * x.
__device__ __forceinline__ void ip_acc(DF& acc, float q, float x) {
    float pe;
    float p = two_prod(q, x, pe);
    float t;
    acc.hi = two_sum(acc.hi, p, t);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, pe));
}

__device__ __forceinline__ void ip_acc2(DF& acc, float q, float xh, float xl) {
    float pe;
    float p = two_prod(q, xh, pe);
    pe = __fmaf_rn(q, xl, pe);
    float t;
    acc.hi = two_sum(acc.hi, p, t);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, pe));
}

// The same transformations on two independent sums at once, with packed
// FP32x2 operations (each half rounds exactly like the scalar operation);
// a - b is written as fma(b, -1, a), one rounding.
struct DF2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2& e) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bv = sub2(s, a);
    const float2 av = sub2(s, bv);
    e = __fadd2_rn(sub2(a, av), sub2(b, bv));
    return s;
}

// acc += (q - x)^2 per half, as l2_acc: q - x = d + e exactly (TwoSum with
// b = -x), d * d = p + pe exactly (with -pe = p - d * (-d) from one FMA, since
// -d = x - q exactly), e^2 dropped.
__device__ __forceinline__ void l2_acc_x2(DF2& acc, float2 q, float2 x) {
    const float2 d = sub2(q, x);
    const float2 bv = sub2(d, q);
    const float2 av = sub2(d, bv);
    const float2 e = sub2(sub2(q, av), __fadd2_rn(x, bv));
    const float2 p = __fmul2_rn(d, d);
    const float2 npe = __ffma2_rn(d, sub2(x, q), p);
    float2 t;
    acc.hi = two_sum2(acc.hi, p, t);
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(t, sub2(__fmul2_rn(__fadd2_rn(d, d), e), npe)));
}

// acc += q * x per half, as ip_acc.
__device__ __forceinline__ void ip_acc_x2(DF2& acc, float2 q, float2 x) {
    const float2 p = __fmul2_rn(q, x);
    const float2 pe = __ffma2_rn(q, x, make_float2(-p.x, -p.y));
    float2 t;
    acc.hi = two_sum2(acc.hi, p, t);
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(t, pe));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float e;
    float s = two_sum(a.hi, b.hi, e);
    float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    float hi = __fadd_rn(s, lo);
    DF r;
    r.lo = __fsub_rn(lo, __fsub_rn(hi, s));
    r.hi = hi;
    return r;
}

__device__ __forceinline__ DF df_shfl_xor(DF v, int m) {
    DF r;
    r.hi = __shfl_xor_sync(kFull, v.hi, m);
    r.lo = __shfl_xor_sync(kFull, v.lo, m);
    return r;
}

// One rounding of hi + lo; the inner-product metric reports -<q, x>.
__device__ __forceinline__ float df_finish(DF a, int metric) {
    float r = __fadd_rn(a.hi, a.lo);
    if (metric == 1) r = -r;
    return r == 0.0f ? 0.0f : r;  // -0 -> +0
}

// ------------------------------------------------------- number formats --

__device__ __forceinline__ float bf16_to_f32(uint32_t h) { return __uint_as_float(h << 16); }

// Four E4M3 codes (one 32-bit word, first code in the low byte) -> FP32,
// exactly, through the hardware pair conversion to FP16 (E4M3 is a subset).
__device__ __forceinline__ void e4m3x4_to_f32(uint32_t wv, float (&x)[4]) {
    const __half2_raw a = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(wv & 0xFFFFu), __NV_E4M3);
    const __half2_raw b = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(wv >> 16), __NV_E4M3);
    x[0] = __half2float(__ushort_as_half(a.x));
    x[1] = __half2float(__ushort_as_half(a.y));
    x[2] = __half2float(__ushort_as_half(b.x));
    x[3] = __half2float(__ushort_as_half(b.y));
}

// ------------------------------------------------------------------ keys --
// A candidate is a 64-bit key: the FP32 distance mapped to an order-preserving
// unsigned integer in the high word, (id << 1 | checked) in the low word, so
// that integer order is (distance, id) order.

__device__ __forceinline__ uint32_t orderable(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float from_orderable(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ uint64_t make_key(float dist, int32_t id) {
    return (uint64_t(orderable(dist)) << 32) | (uint64_t(uint32_t(id)) << 1);
}

__device__ __forceinline__ int32_t key_id(uint64_t k) { return int32_t(uint32_t(k) >> 1); }
__device__ __forceinline__ float key_dist(uint64_t k) { return from_orderable(uint32_t(k >> 32)); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Ascending bitonic sort of one key per lane across the warp.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t o = __shfl_xor_sync(kFull, v, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            v = (lower == up) ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}

// ------------------------------------------------- bulk copies (TMA unit) --
// One cp.async.bulk per gathered row, completing on a per-warp mbarrier by
// transaction bytes; the warp waits on the barrier's phase parity.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Shared memory that generic loads have read may be overwritten by the next
// bulk copies only after this fence.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// L2 cache policies: rows that many queries reuse (the reduced rows, the
// subgraph) are kept with evict_last; the full rows and the full graph, which
// exceed L2, stream through with evict_first so that they do not displace them.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// bulk_copy_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_copy_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                   uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
// Read-only 32-bit load with an L2 cache policy.
__device__ __forceinline__ int32_t ld_nc_hint(const int32_t* p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// One 32-byte global load (a 256-bit vector access, one instruction instead of
// two 128-bit ones); p must be 32-byte aligned.  Ordered after earlier stores
// of the warp by the caller's __syncwarp.
__device__ __forceinline__ void ld_global_32B(const void* p, uint4& x, uint4& y) {
    asm volatile("ld.global.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(x.x), "=r"(x.y), "=r"(x.z), "=r"(x.w), "=r"(y.x), "=r"(y.y), "=r"(y.z), "=r"(y.w)
                 : "l"(p)
                 : "memory");
}

// Wait until the barrier completes the phase with the given parity.  Gives up
// after max_iter polls and returns false (the caller reports an error).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace pilot
