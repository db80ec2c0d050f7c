// search_impl.cuh -- the staged search kernels (Sec. 4.1 stages (1)-(3),
// Alg. 1), included by one translation unit per reduced-row type
// (search_f32.cu, search_bf16.cu, search_fp8.cu) so that they compile in
// parallel; search.cu holds the dispatch and the host-side helpers.
//
//
// A persistent kernel: every warp repeatedly takes the next query and runs,
// with all per-query state in its slice of shared memory,
//   FES check     exact distances of the FES survivors, certified against the
//                 scoring bound, else an exact scan of the entry set (Sec. 5)
//   stage (1)     Algorithm 1 on the subgraph with reduced rows (Sec. 4.1 (1))
//   re-rank       full-vector distances of stage (1)'s candidates; a fresh
//                 visited set holding exactly them (Sec. 4.1 (2))
//   stage (2)     `stage2_expansions` expansions on the subgraph with full rows
//   stage (3)     Algorithm 1 on the full graph with full rows, all candidates
//                 unchecked, reusing stage (2)'s visited set (Sec. 4.1 (3))
//   output        the first k candidates by (distance, id)
//
// Per-warp shared memory: the candidate list C (sorted 64-bit keys), the
// query and projected query, and a staging buffer for gathered rows.  The
// visited sets live in HBM: one open-addressing hash table of 16-bit entries
// per warp slot, sized by ef and the degree (not by n), whose bucket headers
// carry an epoch tag so that a new set costs one epoch step.  An expansion
// probes the table for all of the expanded node's neighbours at once (one
// 32-byte bucket per lane).  In stage (1) every neighbour's reduced row is
// copied into shared memory while the probe runs; in stages (2)(3) only the
// unvisited full rows are copied, after it; each copy is one bulk copy
// completing on the warp's mbarrier.  Once C is full, a plain FP32 pass with
// a rigorous error bound first rejects the rows that cannot enter C (one row
// per lane, or eight lanes per row for few or long rows); only the others get
// the exact (error-free) distance, eight lanes per 128-byte line and a
// shuffle butterfly per row.  Up to three new keys are inserted into C one at
// a time; more are sorted with a warp bitonic sort and merged into C by rank.
#pragma once

#include <cfloat>
#include <climits>

#include "device_common.cuh"
#include "kernels.h"

namespace pilot {
namespace {

constexpr int kCand = 32;   // distance batch (rows)
constexpr int kMaxExpansionsPerStage = 1 << 22;
constexpr uint32_t kMaxPolls = 1u << 24;   // bound on polls of one gather's barrier

struct Layout {
    int pool_cap;      // keys C can hold: ef rounded up to a multiple of 32 (at least 32)
    int off_pool0, off_cand, off_dist, off_bar, off_sel, off_bkeys, off_q, off_qp, off_stage;
    int per_warp;
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Per-warp shared memory: the fixed-size scratch arrays first, at constant
// offsets from the warp's base (so that addressing them needs no registers of
// their own), then the candidate list, the query rows and the staging buffer.
constexpr int kOffCand = 0, kOffDist = kCand * 4, kOffSel = kCand * 8, kOffBkeys = kCand * 12,
              kOffBar = kCand * 20, kOffPool = kCand * 20 + 16;

__host__ __device__ inline Layout make_layout(const DevIndex& ix, const SearchConfig& cfg) {
    Layout L;
    L.pool_cap = round_up(cfg.ef < 32 ? 32 : cfg.ef, 32);
    int o = kOffPool + L.pool_cap * 8;
    L.off_pool0 = kOffPool;
    L.off_cand = kOffCand;
    L.off_dist = kOffDist;
    L.off_bar = kOffBar;
    L.off_sel = kOffSel;
    L.off_bkeys = kOffBkeys;
    o = round_up(o, 16);
    L.off_q = o; o += ix.d_pad * 4;
    L.off_qp = o; o += ix.qp_pad * 4;
    o = round_up(o, 128);
    L.off_stage = o; o += cfg.stage_bytes;
    L.per_warp = round_up(o, 128);
    return L;
}

struct Warp {
    uint8_t* base;       // this warp's slice of shared memory
    int32_t nx_tag;      // whose adjacency row nx_v0 holds: u (view 3), ~u (view 1), INT_MIN none
    int32_t nx_v0;       // entry `lane` of that row
    __device__ __forceinline__ uint64_t* pool() const { return reinterpret_cast<uint64_t*>(base + kOffPool); }
    __device__ __forceinline__ int32_t* cand() const { return reinterpret_cast<int32_t*>(base + kOffCand); }
    __device__ __forceinline__ int32_t* sel() const { return reinterpret_cast<int32_t*>(base + kOffSel); }
    __device__ __forceinline__ float* dist() const { return reinterpret_cast<float*>(base + kOffDist); }
    __device__ __forceinline__ uint64_t* bkeys() const { return reinterpret_cast<uint64_t*>(base + kOffBkeys); }
    __device__ __forceinline__ uint64_t* bar() const { return reinterpret_cast<uint64_t*>(base + kOffBar); }
    uint16_t* vis;       // this warp slot's visited table
    uint32_t vis_mask;   // buckets in use - 1
    int vis_qbits;       // quotient bits of an entry
    int id_bits;
    int overflow;        // insertions that found no room (visited again if met again)
    float* q;
    float* qp;
    uint8_t* stage;
    int S;          // candidates in C
    int ef;         // this query's list size
    int lb;         // every candidate before position lb is checked
    uint32_t epoch_ctr;
    uint32_t epoch;  // 1..kVisEpochs: the current set's bucket-header tag
    int lane;
    const uint8_t* red_base;   // the reduced rows (kept in L2 by a cache policy)
    uint32_t phase;     // parity of the barrier phase being waited for
    bool failed;        // a gather did not complete within kMaxPolls polls
#ifdef PILOT_CHECKED
    int32_t* status;    // status words: [6] counts out-of-range indices skipped (checked build)
#endif
};

// ------------------------------------------------------------ visited set --
// Node v is mapped by h, a bijection of [0, 2^id_bits) (multiply by an odd
// constant, xor-shift, multiply: each step is invertible on id_bits bits), to
// its home bucket, the top bits of h, and its quotient s, the low vis_qbits
// bits.  The pair (bucket, s) identifies v, so an entry holds only s and the
// probe r at which v was placed, home + r: (s << 3) | (r + 1), never zero.
// Bucket layout (16 words, one 32-byte sector): word 0 = epoch << 4 | count,
// words 1..count the entries.  A bucket is zeroed when it is first written in
// an epoch, so the words past its count are zero and a lookup may compare
// all 15 without masking.
__device__ __forceinline__ uint32_t vis_hash(uint32_t v, int bits) {
    const uint32_t m = bits >= 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
    uint32_t h = (v * 0x9E3779B1u) & m;
    h ^= h >> ((bits + 1) >> 1);
    return (h * 0x85EBCA77u) & m;
}

// Nonzero when some 16-bit half of x is zero (a borrow out of a zero low half
// can only flag the high half as well, so the test is exact as an "any").
__device__ __forceinline__ uint32_t zero_half(uint32_t x) { return (x - 0x00010001u) & ~x & 0x80008000u; }

// Probe-and-insert of node v for every lane with `valid`: returns true when v
// is not yet in the current set, and records it.  Lanes probe their bucket in
// parallel; lanes that need room in the same bucket take its free entries in
// lane order (the first of them also writes the header, zeroing a bucket of
// an older epoch first), and those left without one move on to the next
// bucket (linear probing).  Counts only grow within a set, so a bucket with
// room ends the search for v.  The valid lanes' ids must be distinct.  An
// insertion that finds no room within kVisMaxProbe buckets reports v as new
// without recording it; if v is met again it is scored again, and the merge
// drops its equal key, so results are unchanged (only the distance counter
// grows).
__device__ __forceinline__ bool visit(Warp& w, int32_t v, bool valid) {
    const uint32_t h = valid ? vis_hash(uint32_t(v), w.id_bits) : 0u;
    uint32_t b = h >> w.vis_qbits;
    const uint32_t s3 = (h & ((1u << w.vis_qbits) - 1u)) << 3;
    bool pending = valid, isnew = false;
#pragma unroll 1
    for (int r = 0; r < kVisMaxProbe; ++r) {
        if (!__any_sync(kFull, pending)) break;
        uint16_t* bp = w.vis + size_t(b) * kVisBucket;
        int cnt = 0;
        bool stale = false;
        if (pending) {
            uint4 x, y;
            ld_global_32B(bp, x, y);
            stale = ((x.x & 0xFFFFu) >> 4) != w.epoch;
            if (!stale) {
                cnt = int(x.x & 15u);
                const uint32_t t2 = (s3 | uint32_t(r + 1)) * 0x10001u;
                // word 0's low half is the header: forced nonzero, never a match
                const uint32_t z = zero_half((x.x ^ t2) | 0x8000u) | zero_half(x.y ^ t2) | zero_half(x.z ^ t2) |
                                   zero_half(x.w ^ t2) | zero_half(y.x ^ t2) | zero_half(y.y ^ t2) |
                                   zero_half(y.z ^ t2) | zero_half(y.w ^ t2);
                if (z) pending = false;
            }
        }
        const unsigned peers = __match_any_sync(kFull, pending ? b : (0x80000000u | unsigned(w.lane)));
        const int rank = __popc(peers & lanemask_lt());
        const int room = (kVisBucket - 1) - cnt;
        if (pending && rank == 0 && room > 0) {
            const int np = __popc(peers);
            const uint32_t hdr = (w.epoch << 4) | uint32_t(cnt + (np < room ? np : room));
            if (stale) {
                uint4* q = reinterpret_cast<uint4*>(bp);
                q[0] = make_uint4(hdr, 0u, 0u, 0u);
                q[1] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                bp[0] = uint16_t(hdr);
            }
        }
        __syncwarp();
        if (pending) {
            if (rank < room) {
                bp[1 + cnt + rank] = uint16_t(s3 | uint32_t(r + 1));
                pending = false;
                isnew = true;
            } else {
                b = (b + 1) & w.vis_mask;
            }
        }
        __syncwarp();
    }
    if (pending) {   // no room: treated as new, not recorded
        isnew = true;
        w.overflow += 1;
    }
    return isnew;
}

// Checked builds (-DPILOT_CHECKED) test every index read from the graph
// before it addresses a row; an out-of-range index is counted in status
// word 6 and skipped instead of being dereferenced.
#ifdef PILOT_CHECKED
#define PILOT_CHECK_INDEX(w, v, limit)                                        \
    do {                                                                     \
        if ((v) >= (limit)) {                                                \
            if ((w).status) atomicAdd(&(w).status[6], 1);                    \
            (v) = -1;                                                        \
        }                                                                    \
    } while (0)
#else
#define PILOT_CHECK_INDEX(w, v, limit) \
    do {                               \
    } while (0)
#endif

// Exact accumulation of one 16-byte chunk of a row into acc: the chunk holds
// 4 FP32, 8 BF16 or 16 FP8 elements; qc points at the matching query elements;
// sc is the row's FP8 scale.
template <int DT, int METRIC>
__device__ __forceinline__ void exact_chunk(DF& acc, uint4 v, const float* qc, float sc) {
    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
    if (DT == 0) {
        const float4 qv = *reinterpret_cast<const float4*>(qc);
        const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (METRIC == 0) l2_acc(acc, qa[e], __uint_as_float(wv[e]));
            else ip_acc(acc, qa[e], __uint_as_float(wv[e]));
        }
    } else if (DT == 1) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 qv = *reinterpret_cast<const float2*>(qc + h * 2);
            const float x0 = bf16_to_f32(wv[h] & 0xFFFFu), x1 = bf16_to_f32(wv[h] >> 16);
            if (METRIC == 0) {
                l2_acc(acc, qv.x, x0);
                l2_acc(acc, qv.y, x1);
            } else {
                ip_acc(acc, qv.x, x0);
                ip_acc(acc, qv.y, x1);
            }
        }
    } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float4 qv = *reinterpret_cast<const float4*>(qc + h * 4);
            const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
            float c[4];
            e4m3x4_to_f32(wv[h], c);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (METRIC == 0) {
                    float xl;
                    const float xh = two_prod(c[b], sc, xl);   // code * scale = xh + xl exactly
                    l2_acc2(acc, qa[b], xh, xl);
                } else {
                    ip_acc(acc, qa[b], c[b]);   // sum q * code; the row's scale is applied once at the end
                }
            }
        }
    }
}

// ---------------------------------------------------- certified pre-filter --
// A plain FP32 evaluation of a row's distance with a rigorous bound on its
// rounding error gives a lower bound lb on the exact distance.  Once C is
// full, a row with lb > nextup(worst distance in C) has an exact FP32 distance
// above the worst one, so the exact path would reject it too; only the other
// rows need the (costlier) error-free evaluation.  With u = 2^-24 and n terms
// (any summation order, every FMA or add rounding once):
//   L2  a = sum fl(q - x)^2:  |fl(q - x) - (q - x)| <= u |q - x| and the sum of
//       non-negative terms carries at most gamma_n relative error, so
//       exact >= a (1 - (n + 3) u (1 + eps));
//   IP  a = sum q x, b = sum |q| |x| (both FMA chains): |a - sum q x| <= gamma_n
//       sum |q x| <= gamma_n b / (1 - gamma_n), so -sum q x >= -a - n u b (1 + eps);
//       FP8 rows: a and b over the codes, times the row's scale s > 0.
// The kernel uses 2 (n + 8) u, twice these constants, rounds toward the safe
// side and subtracts 1e-36 for underflow (at most n * 2^-150 in all).  The
// bounds hold for any order of summation, so lanes may combine partial sums
// in any pattern.
// FP8 rows under L2 (code x scale rounded before the subtraction) are always
// scored exactly.
constexpr float kTiny = 1e-36f;

// Plain FP32 accumulation of one 16-byte chunk of a row into two partial
// sums a.x, a.y (alternate elements, one packed FP32x2 operation per pair;
// each half rounds exactly like its scalar counterpart) and, for the inner
// product, the sum of |q| |x| into b.
template <int DT, int METRIC>
__device__ __forceinline__ void approx_chunk(float2& a, float& b, uint4 v, const float* qc) {
    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
    float x[16], qa[16];
    constexpr int E = DT == 0 ? 4 : (DT == 1 ? 8 : 16);
    if (DT == 0) {
        const float4 qv = *reinterpret_cast<const float4*>(qc);
        qa[0] = qv.x; qa[1] = qv.y; qa[2] = qv.z; qa[3] = qv.w;
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = __uint_as_float(wv[e]);
    } else if (DT == 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 qv = *reinterpret_cast<const float4*>(qc + h * 4);
            qa[h * 4 + 0] = qv.x; qa[h * 4 + 1] = qv.y; qa[h * 4 + 2] = qv.z; qa[h * 4 + 3] = qv.w;
        }
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            x[2 * h] = bf16_to_f32(wv[h] & 0xFFFFu);
            x[2 * h + 1] = bf16_to_f32(wv[h] >> 16);
        }
    } else {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float4 qv = *reinterpret_cast<const float4*>(qc + h * 4);
            qa[h * 4 + 0] = qv.x; qa[h * 4 + 1] = qv.y; qa[h * 4 + 2] = qv.z; qa[h * 4 + 3] = qv.w;
            float c[4];
            e4m3x4_to_f32(wv[h], c);   // inner product over the codes; the scale comes after
            x[h * 4 + 0] = c[0]; x[h * 4 + 1] = c[1]; x[h * 4 + 2] = c[2]; x[h * 4 + 3] = c[3];
        }
    }
    const float2 neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int e = 0; e < E; e += 2) {
        const float2 qq = make_float2(qa[e], qa[e + 1]), xx = make_float2(x[e], x[e + 1]);
        if (METRIC == 0) {
            const float2 t = __ffma2_rn(xx, neg1, qq);   // fl(q - x) per half: -x is exact
            a = __ffma2_rn(t, t, a);
        } else {
            a = __ffma2_rn(qq, xx, a);
            b = __fmaf_rn(fabsf(qa[e]), fabsf(x[e]), b);
            b = __fmaf_rn(fabsf(qa[e + 1]), fabsf(x[e + 1]), b);
        }
    }
}

// Keep flags of staged rows rows(0..m-1): w.sel()[i] = 0 when row rows(i)'s
// certified lower bound exceeds thr (it cannot enter C), else 1.  One row per
// lane: lane i sums its whole row (the staging stride keeps the lanes' chunks
// in distinct banks), so no shuffle is needed; cand[cand_off + row] is the
// row's id (for the FP8 scale).  The caller synchronises the warp afterwards.
// Certified lower bound on the exact distance of one staged row (rowp, n_elems
// elements); sc is the row's FP8 scale (inner product only).
template <int DT, int METRIC>
__device__ __forceinline__ float approx_lb(const uint8_t* rowp, int row_bytes, const float* q, int n_elems,
                                           const float* __restrict__ sc_ptr) {
    constexpr int EPC = DT == 0 ? 4 : (DT == 1 ? 8 : 16);
    const int nch = row_bytes >> 4;
    float2 a = make_float2(0.0f, 0.0f);
    float b = 0.0f;
#pragma unroll 2
    for (int c = 0; c < nch; ++c)
        approx_chunk<DT, METRIC>(a, b, *reinterpret_cast<const uint4*>(rowp + c * 16), q + c * EPC);
    const float A = __fadd_rn(a.x, a.y);
    const float rel = float(n_elems + 8) * 1.1920928955078125e-7f;   // 2 (n + 8) u, u = 2^-24
    if (METRIC == 0) return __fsub_rd(__fmaf_rd(A, -rel, A), kTiny);
    if (DT == 2) {
        const float sc = __ldg(sc_ptr);
        return __fsub_rd(-__fmul_ru(sc, __fmaf_ru(rel, b, A)), kTiny);
    }
    return __fsub_rd(__fmaf_rd(-rel, b, -A), kTiny);
}

template <int DT, int METRIC, class Rows>
__device__ __forceinline__ void approx_keep(Warp& w, int row_bytes, const float* __restrict__ scales,
                                            const float* q, int m, int cand_off, int n_elems, float thr,
                                            Rows rows) {
    const int i = w.lane;
    if (i >= m) return;
    const int row = rows(i);   // the staged row lane i tests
    const float lb = approx_lb<DT, METRIC>(w.stage + row * stage_stride(row_bytes), row_bytes, q, n_elems,
                                           DT == 2 ? scales + w.cand()[cand_off + row] : nullptr);
    w.sel()[i] = lb > thr ? 0 : 1;
}

// Keep flags like approx_keep for FP32 rows, eight lanes per row: lane
// (g, mm) sums chunks mm + 8 t of staged row g + 4 j, four rows at a time, and
// a butterfly over the row's eight lanes adds the partial sums (the bound
// holds for any summation order).  Rows are whole 128-byte lines, so every
// lane of a row has the same number of chunks.
template <int METRIC>
__device__ __forceinline__ void approx_keep8(Warp& w, int row_bytes, const float* q, int m, int n_elems, float thr) {
    const int g = w.lane >> 3, mm = w.lane & 7;
    const int nch = row_bytes >> 4;
    const float rel = float(n_elems + 8) * 1.1920928955078125e-7f;   // 2 (n + 8) u, u = 2^-24
#pragma unroll 1
    for (int j = 0; j < ((m + 3) >> 2); ++j) {
        const int i = g + 4 * j;
        const uint8_t* rowp = w.stage + (i < m ? i : 0) * stage_stride(row_bytes);
        float2 a = make_float2(0.0f, 0.0f);
        float b = 0.0f;
#pragma unroll 2
        for (int c = mm; c < nch; c += 8)
            approx_chunk<0, METRIC>(a, b, *reinterpret_cast<const uint4*>(rowp + c * 16), q + c * 4);
        float A = __fadd_rn(a.x, a.y);
        A = __fadd_rn(A, __shfl_xor_sync(kFull, A, 1));
        A = __fadd_rn(A, __shfl_xor_sync(kFull, A, 2));
        A = __fadd_rn(A, __shfl_xor_sync(kFull, A, 4));
        float lb;
        if (METRIC == 0) {
            lb = __fsub_rd(__fmaf_rd(A, -rel, A), kTiny);
        } else {
            b = __fadd_rn(b, __shfl_xor_sync(kFull, b, 1));
            b = __fadd_rn(b, __shfl_xor_sync(kFull, b, 2));
            b = __fadd_rn(b, __shfl_xor_sync(kFull, b, 4));
            lb = __fsub_rd(__fmaf_rd(-rel, b, -A), kTiny);
        }
        if (mm == 0 && i < m) w.sel()[i] = lb > thr ? 0 : 1;
    }
}

// Exact distances of the staged rows sel(i), i < m, into dist[sel(i)].
// Staged row s lives at stage + s * stage_stride(row_bytes).  Lane (g, mm) covers chunks
// mm + 8 t of rows g + 4 j; one row slot j at a time (a warp-uniform loop,
// kept compact so that the search's inner loop stays in the instruction
// cache), the eight lanes of a row combining their pairs by a butterfly.
// df_add is symmetric, so every lane of the row ends with the same sum.
template <int DT, int METRIC, class Sel>
__device__ __forceinline__ void exact_staged(Warp& w, int row_bytes, const float* __restrict__ scales,
                                             const float* q, int m, Sel sel, int cand_off) {
    const int g = w.lane >> 3, mm = w.lane & 7;
    const int F8 = row_bytes >> 7;
    constexpr int EPC = DT == 0 ? 4 : (DT == 1 ? 8 : 16);
    const int jrows = (m + 3) >> 2;
#pragma unroll 1
    for (int j = 0; j < jrows; ++j) {
        const int i = g + 4 * j;
        const bool ok = i < m;
        const int srow = sel(ok ? i : 0);
        const uint8_t* rowp = w.stage + srow * stage_stride(row_bytes);
        const float sc = DT == 2 ? __ldg(scales + w.cand()[cand_off + srow]) : 1.0f;
        DF acc{0.0f, 0.0f};
        if constexpr (DT == 0) {
            // FP32 rows: elements (0, 1) and (2, 3) of each chunk in the two
            // halves of packed pairs, the halves added at the end
            DF2 a2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll 1
            for (int t = 0; t < F8; ++t) {
                const int c = mm + 8 * t;
                const float4 xv = *reinterpret_cast<const float4*>(rowp + c * 16);
                const float4 qv = *reinterpret_cast<const float4*>(q + c * 4);
                if (METRIC == 0) {
                    l2_acc_x2(a2, make_float2(qv.x, qv.y), make_float2(xv.x, xv.y));
                    l2_acc_x2(a2, make_float2(qv.z, qv.w), make_float2(xv.z, xv.w));
                } else {
                    ip_acc_x2(a2, make_float2(qv.x, qv.y), make_float2(xv.x, xv.y));
                    ip_acc_x2(a2, make_float2(qv.z, qv.w), make_float2(xv.z, xv.w));
                }
            }
            acc = df_add(DF{a2.hi.x, a2.lo.x}, DF{a2.hi.y, a2.lo.y});
        } else {
#pragma unroll 1
            for (int t = 0; t < F8; ++t) {
                const int c = mm + 8 * t;
                exact_chunk<DT, METRIC>(acc, *reinterpret_cast<const uint4*>(rowp + c * 16), q + c * EPC, sc);
            }
        }
        acc = df_add(acc, df_shfl_xor(acc, 1));
        acc = df_add(acc, df_shfl_xor(acc, 2));
        acc = df_add(acc, df_shfl_xor(acc, 4));
        if (DT == 2 && METRIC == 1) {
            // sum q_e (c_e s) = s * sum q_e c_e exactly; scale the pair once
            float e;
            const float p = two_prod(acc.hi, sc, e);
            acc = DF{p, __fmaf_rn(acc.lo, sc, e)};
        }
        if (ok && mm == 0) w.dist()[cand_off + srow] = df_finish(acc, METRIC);
    }
}

// Gather rows cand[r0..r1) (r1 - r0 <= 32) into the staging buffer: lane i
// issues one bulk copy of row r0 + i; all complete on the warp's mbarrier.
// Rows in host memory mapped into the device's address space (`plain`) are
// copied instead with 16-byte loads spread over all lanes.
// Rows in pinned host memory mapped into the device's address space: 16-byte
// loads spread over the lanes, 4 independent loads in flight per lane before
// any is stored (the host link's latency is what this waits on; more would
// push the kernel's register allocation past 128 and spill).
__device__ __noinline__ void gather_rows_plain(uint8_t* stage, const uint8_t* __restrict__ base, int row_bytes,
                                              const int32_t* cand, int n, int lane) {
    constexpr int kInFlight = 4;
    const int cpr = row_bytes >> 4;
    const int total = n * cpr;
    __syncwarp();
    for (int c0 = lane; c0 < total; c0 += 32 * kInFlight) {
        uint4 v[kInFlight];
#pragma unroll
        for (int u = 0; u < kInFlight; ++u) {
            const int c = c0 + 32 * u;
            if (c < total) {
                const int r = c / cpr, o = c - r * cpr;
                v[u] = *reinterpret_cast<const uint4*>(base + int64_t(cand[r]) * row_bytes + o * 16);
            }
        }
#pragma unroll
        for (int u = 0; u < kInFlight; ++u) {
            const int c = c0 + 32 * u;
            if (c < total) {
                const int r = c / cpr, o = c - r * cpr;
                *reinterpret_cast<uint4*>(stage + r * stage_stride(row_bytes) + o * 16) = v[u];
            }
        }
    }
    __syncwarp();
}

// Issue one bulk copy per row for rows cand[r0 .. r0+n) (n <= 32) into the
// staging buffer, all completing on the warp's mbarrier; gather_wait waits.
__device__ __forceinline__ void gather_issue(Warp& w, const uint8_t* __restrict__ base, int row_bytes, int r0,
                                             int n) {
    fence_proxy_async_smem();
    __syncwarp();
    if (w.lane == 0) mbar_arrive_expect_tx(w.bar(), uint32_t(n * row_bytes));
    __syncwarp();
    if (w.lane < n) {
        // reduced rows (small, reused across queries) stay in L2; full rows stream
        const uint64_t pol = base == w.red_base ? l2_evict_last_policy() : l2_evict_first_policy();
        bulk_copy_g2s_hint(w.stage + w.lane * stage_stride(row_bytes),
                           base + int64_t(w.cand()[r0 + w.lane]) * row_bytes, uint32_t(row_bytes), w.bar(), pol);
    }
}

// Copy row v (of `base`, row_bytes each) into staging slot `lane` for every
// lane with v >= 0 (the lanes of mask vb), completing on the warp's barrier;
// the rows are kept in L2 (evict_last).  gather_wait waits.
__device__ __forceinline__ void gather_issue_lanes(Warp& w, const uint8_t* __restrict__ base, int row_bytes, int32_t v,
                                                   unsigned vb) {
    fence_proxy_async_smem();
    __syncwarp();
    if (w.lane == 0) mbar_arrive_expect_tx(w.bar(), uint32_t(__popc(vb) * row_bytes));
    __syncwarp();
    if (v >= 0)
        bulk_copy_g2s_hint(w.stage + w.lane * stage_stride(row_bytes), base + int64_t(v) * row_bytes,
                           uint32_t(row_bytes), w.bar(), l2_evict_last_policy());
}

__device__ __forceinline__ void gather_wait(Warp& w) {
    if (!mbar_wait(w.bar(), w.phase, kMaxPolls)) {
        // give the copies still in flight one more bounded wait, then report
        mbar_wait(w.bar(), w.phase, kMaxPolls);
        w.failed = true;
    }
    w.phase ^= 1u;
    __syncwarp();
}

__device__ __forceinline__ void gather_rows(Warp& w, const uint8_t* __restrict__ base, int row_bytes, int r0, int r1,
                                            bool plain) {
    const int n = r1 - r0;
    if (plain) {   // host memory: out of line, off the device-resident path
        gather_rows_plain(w.stage, base, row_bytes, w.cand() + r0, n, w.lane);
        return;
    }
    gather_issue(w, base, row_bytes, r0, n);
    gather_wait(w);
}

// Exact distances of rows cand[0..m) of a row array (`base`, `row_bytes` per
// row, element type DT: 0 f32, 1 bf16, 2 fp8 codes with per-row `scales`) to
// the query q in shared memory, into dist[0..m).  Rows are gathered with one
// bulk copy each, P at a time (as many as the staging buffer holds).
template <int DT, int METRIC>
__device__ __forceinline__ void batch_dist(Warp& w, const uint8_t* __restrict__ base, int row_bytes,
                                           const float* __restrict__ scales, const float* q, int m,
                                           int stage_bytes, bool plain) {
    int P = stage_bytes / stage_stride(row_bytes);
    P = P >= kCand ? kCand : (P & ~3);
    for (int r0 = 0; r0 < m; r0 += P) {
        const int r1 = r0 + P < m ? r0 + P : m;
        gather_rows(w, base, row_bytes, r0, r1, plain);
        exact_staged<DT, METRIC>(w, row_bytes, scales, q, r1 - r0, [](int i) { return i; }, r0);
        __syncwarp();
    }
}

// Distances of rows cand[0..m) like batch_dist, for an expansion whose list
// may be full: with `filter`, rows whose certified lower bound exceeds thr get
// +inf (they cannot enter C) and only the others are scored exactly.
template <int DT, int METRIC>
__device__ __forceinline__ void filtered_dist(Warp& w, const uint8_t* __restrict__ base, int row_bytes,
                                              const float* __restrict__ scales, const float* q, int m,
                                              int stage_bytes, bool plain, bool filter, float thr, int n_elems) {
    int P = m;   // one pass when the staging buffer holds every row (no division on this path)
    if (m * stage_stride(row_bytes) > stage_bytes) {
        P = stage_bytes / stage_stride(row_bytes);
        P = P >= kCand ? kCand : (P & ~3);
    }
    for (int r0 = 0; r0 < m; r0 += P) {
        const int r1 = r0 + P < m ? r0 + P : m;
        const int nr = r1 - r0;
        gather_rows(w, base, row_bytes, r0, r1, plain);
        bool keep = w.lane < nr;
        if (filter) {
            // one row per lane, or eight lanes per row when a row per lane
            // would leave most lanes idle (few or long rows): the cost of
            // each, in chunk steps, is nch against ceil(nr / 4) (nch / 8 + ~1.4)
            const int nch = row_bytes >> 4;
            if (DT == 0 && ((nr + 3) >> 2) * (nch + 11) < nch * 8)
                approx_keep8<METRIC>(w, row_bytes, q, nr, n_elems, thr);
            else
                approx_keep<DT, METRIC>(w, row_bytes, scales, q, nr, r0, n_elems, thr, [](int i) { return i; });
            __syncwarp();
            keep = keep && w.sel()[w.lane] != 0;
            __syncwarp();
        }
        // staged rows still to score exactly, listed in w.sel()
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) w.sel()[__popc(km & lanemask_lt())] = w.lane;
        else if (w.lane < nr) w.dist()[r0 + w.lane] = INFINITY;
        __syncwarp();
        const int m2 = __popc(km);
        if (m2 > 0) exact_staged<DT, METRIC>(w, row_bytes, scales, q, m2, [&](int i) { return w.sel()[i]; }, r0);
        __syncwarp();
    }
}

// The nkeep (<= 8) keys held by some lanes (kKeyEmpty elsewhere), sorted
// into lanes 0..nkeep-1: each key's rank is counted against the others (the
// keys are distinct), cheaper than the 32-lane sorting network for a few keys.
__device__ __forceinline__ uint64_t place_few(Warp& w, uint64_t key, int nkeep) {
    const bool has = key != kKeyEmpty;
    const unsigned hm = __ballot_sync(kFull, has);
    if (has) w.bkeys()[__popc(hm & lanemask_lt())] = key;
    __syncwarp();
    int rank = 0;
    for (int j = 0; j < nkeep; ++j) rank += w.bkeys()[j] < key;
    __syncwarp();
    if (has) w.bkeys()[rank] = key;
    __syncwarp();
    const uint64_t out = w.lane < nkeep ? w.bkeys()[w.lane] : kKeyEmpty;
    __syncwarp();
    return out;
}

// Insert one new key (every lane holds it) into C, the common case once C is
// full (a few keys are inserted one at a time: C stays sorted and keeps the ef
// best of the union, as the merge does).  Its lower bound comes from two ballots, over the chunk heads C[32 i]
// and then over the chunk that holds it; a key equal to one in C is dropped.
// The tail C[p .. Snew - 2] moves up one position, two 32-slot chunks per
// step from the last: every lane reads its sources before any lane writes,
// and a step writes no position that a later step reads.
__device__ __forceinline__ void insert_one(Warp& w, uint64_t key, int ef) {
    const int lane = w.lane;
    uint64_t* A = w.pool();
    const int S = w.S;
    const int h = lane << 5;
    const unsigned hb = __ballot_sync(kFull, h < S && (A[h] & ~1ull) < key);   // a prefix: C is sorted
    int p = 0;
    if (hb) {
        const int c = 31 - __clz(hb);
        const int i = (c << 5) + lane;
        p = (c << 5) + __popc(__ballot_sync(kFull, i < S && (A[i] & ~1ull) < key));
    }
    const int Snew = min(S + 1, ef);
    if (p >= Snew || (p < S && (A[p] & ~1ull) == key)) return;
    for (int c = (Snew - 1) >> 5; c >= (p >> 5); c -= 2) {
        const int i0 = (c << 5) + lane, i1 = i0 - 32;
        const bool m0 = i0 > p && i0 < Snew, m1 = i1 > p;
        const uint64_t v0 = m0 ? A[i0 - 1] : 0ull, v1 = m1 ? A[i1 - 1] : 0ull;
        __syncwarp();
        if (m0) A[i0] = v0;
        if (m1) A[i1] = v1;
    }
    __syncwarp();
    if (lane == 0) A[p] = key;
    __syncwarp();
    w.S = Snew;
    if (p < w.lb) w.lb = p;
}

// Merge nb sorted new keys (lanes 0..nb-1, kKeyEmpty beyond) into C in place.
// A new key equal to one already in C (same distance and id) is dropped.  Each
// kept key lands at (its rank among the new keys) + (its lower bound in C);
// output positions are filled from the last 32-slot chunk down to the first
// changed one, every lane reading its source before any lane writes, so an
// element is always read before it is overwritten.  C keeps its ef best.
__device__ __forceinline__ void merge_new(Warp& w, uint64_t key, int nb, int ef) {
    const int lane = w.lane;
    uint64_t* A = w.pool();
    const int S = w.S;
    // lower bound of every new key in C, in lock step (fixed step count)
    int p = 0;
    for (int step = S > 0 ? (1 << (31 - __clz(S))) : 0; step > 0; step >>= 1)
        if (p + step <= S && (A[p + step - 1] & ~1ull) < key) p += step;
    const bool dup = lane < nb && p < S && (A[p] & ~1ull) == key;
    const bool mine = lane < nb && !dup;
    const unsigned keep = __ballot_sync(kFull, mine);
    const int nb2 = __popc(keep);
    if (nb2 == 0) return;
    const int ci = __popc(keep & lanemask_lt());
    const int np = mine ? p + ci : 0x7FFFFFFF;
    if (mine) w.bkeys()[ci] = key;
    const int Snew = min(S + nb2, ef);
    const int lo_pos = __reduce_min_sync(kFull, np);
    __syncwarp();
    if (lo_pos >= Snew) return;
    // two 32-position chunks per step, from the last one down
    const int c_lo = lo_pos >> 5;
    const unsigned upto = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
    for (int c = (Snew - 1) >> 5; c >= c_lo; c -= 2) {
        const bool two = c - 1 >= c_lo;
        const int base0 = c << 5, base1 = base0 - 32;
        const unsigned bit0 = (mine && np >= base0 && np < base0 + 32) ? (1u << (np - base0)) : 0u;
        const unsigned bit1 = (two && mine && np >= base1 && np < base0) ? (1u << (np - base1)) : 0u;
        const unsigned m0 = __reduce_or_sync(kFull, bit0);
        const unsigned m1 = __reduce_or_sync(kFull, bit1);
        const int before0 = __popc(__ballot_sync(kFull, mine && np < base0));
        const int before1 = before0 - __popc(m1);
        const int pos0 = base0 + lane, pos1 = base1 + lane;
        const bool wr0 = pos0 < Snew && pos0 >= lo_pos;
        const bool wr1 = two && pos1 >= lo_pos;
        uint64_t v0 = 0, v1 = 0;
        if (wr0) {
            const int kle = before0 + __popc(m0 & upto);
            v0 = ((m0 >> lane) & 1u) ? w.bkeys()[kle - 1] : A[pos0 - kle];
        }
        if (wr1) {
            const int kle = before1 + __popc(m1 & upto);
            v1 = ((m1 >> lane) & 1u) ? w.bkeys()[kle - 1] : A[pos1 - kle];
        }
        __syncwarp();
        if (wr0) A[pos0] = v0;
        if (wr1) A[pos1] = v1;
        __syncwarp();
    }
    w.S = Snew;
    if (lo_pos < w.lb) w.lb = lo_pos;
}

// Ascending sort of C's S keys in place (the re-rank): a bitonic network
// over the next power of two N >= S in the form whose compare-exchanges all
// put the smaller key first (the first step of each merge pairs i with its
// mirror i ^ (k - 1)), so the positions past S can stand for +inf without
// being stored: a pair reaching past S never swaps.  C needs no more room
// than S keys.
__device__ __forceinline__ void sort_pool(Warp& w) {
    uint64_t* A = w.pool();
    const int S = w.S;
    int N = 1;
    while (N < S) N <<= 1;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int x = j == (k >> 1) ? k - 1 : j;
            for (int i = w.lane; i < S; i += 32) {
                const int l = i ^ x;
                if (l > i && l < S) {
                    const uint64_t a = A[i], b = A[l];
                    if (a > b) {
                        A[i] = b;
                        A[l] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ uint64_t warp_min_key(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t x = __shfl_xor_sync(kFull, v, o);
        v = x < v ? x : v;
    }
    return v;
}

enum Phase : int { kStage1 = 1, kRerank = 2, kStage2 = 3, kStage3 = 4, kDone = 5 };

// Resumable per-query search state (the candidate list itself is in Warp).
struct QState {
    int phase, it;                      // current phase; expansions in it so far
    int e1, d1, e2, d2, e3, d3;         // expansions / distances per stage
    int n_rerank;
    int fallback, capped;
    uint64_t best;                      // FES entry key (compact id)
};

// Start a new visited set for this warp slot.  Epochs cycle through 1..M,
// M = epoch_max <= kVisEpochs (the bucket header's epoch field); before a
// cycle restarts the slot's whole table (stride words) is cleared.
__device__ __forceinline__ void new_visited_set(Warp& w, int64_t stride, uint32_t M) {
    w.epoch_ctr += 1;
    const uint32_t r = M > 1 ? w.epoch_ctr % M : 0u;
    if (r == 0) {
        uint4* p = reinterpret_cast<uint4*>(w.vis);
        const int64_t n16 = stride >> 3;
        for (int64_t i = w.lane; i < n16; i += 32) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    w.epoch = r + 1;
    __syncwarp();
}

// WIDE: reduced rows too wide for 32 staging slots (32 x stage_stride(red) >
// stage_bytes); stage (1) then gathers them after the probe, like full rows.
template <int DT, int METRIC, bool WIDE>
struct Searcher {
    const DevIndex& ix;
    const SearchConfig& cfg;
    Warp& w;

    __device__ __forceinline__ void reduced_batch(int m) {
        batch_dist<DT, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.red), ix.red_row_bytes, ix.red_scales, w.qp,
                               m, cfg.stage_bytes, false);
    }
    __device__ __forceinline__ void full_batch(int m) {
        batch_dist<0, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.full), ix.full_row_bytes, nullptr, w.q, m,
                              cfg.stage_bytes, ix.full_host != 0);
    }
    // Adjacency row of node u in a view (null if it has none).
    __device__ __forceinline__ const int32_t* adjacency(int view, int32_t u) const {
        if (view == 1) return ix.sub_adj + int64_t(u) * ix.R_sub;
        if (view == 2) {
            const int32_t cu = __ldg(ix.full2sub + u);   // every stage (2) candidate is sampled
            return cu < 0 ? nullptr : ix.sub_adj + int64_t(cu) * ix.R_sub;
        }
        return ix.graph + int64_t(u) * ix.R;
    }

    // One step of Algorithm 1.  view 1: subgraph + reduced rows, compact ids;
    // view 2: subgraph + full rows, original ids; view 3: full graph + full
    // rows.  Returns false when C has no unchecked candidate.
    __device__ bool expand(int view, int& n_exp, int& n_dist) {
        const int lane = w.lane;
        int idx = -1, idx2 = -1;
        for (int b0 = w.lb; b0 < w.S; b0 += 32) {
            const int i = b0 + lane;
            const bool unc = i < w.S && !(w.pool()[i] & 1ull);
            const unsigned b = __ballot_sync(kFull, unc);
            if (b) {
                idx = b0 + __ffs(b) - 1;
                const unsigned b2 = b & (b - 1);
                if (b2) idx2 = b0 + __ffs(b2) - 1;
                break;
            }
        }
        if (idx < 0) {
            w.lb = w.S;
            return false;
        }
        const uint64_t key = w.pool()[idx];
        __syncwarp();
        if (lane == 0) w.pool()[idx] = key | 1ull;
        w.lb = idx + 1;
        n_exp += 1;
        const int32_t u = key_id(key);
        const int32_t* row = adjacency(view, u);
        const int W = view == 3 ? ix.R : (row ? ix.R_sub : 0);
        const uint64_t pol = view == 3 ? l2_evict_first_policy() : l2_evict_last_policy();
        // The next expansion most likely takes the second unchecked candidate
        // (the guess fails about 40% of the time): its adjacency row (degree
        // up to 32) is loaded into a register now and used then if the guess
        // held, a one-entry cache of (view, node) -> row.  Stage (2), two
        // expansions reached through full2sub, and wider rows only prefetch
        // the row into L2.
        const bool have = view != 2 && W <= 32 && (view == 3 ? u : ~u) == w.nx_tag;
        const int32_t h0 = w.nx_v0;
        w.nx_tag = INT_MIN;
        if (idx2 >= 0) {
            const int32_t u2 = key_id(w.pool()[idx2]);
            const int32_t* r2 = adjacency(view, u2);
            const int W2 = view == 3 ? ix.R : ix.R_sub;
            if (view != 2 && W2 <= 32) {
                w.nx_v0 = lane < W2 ? ld_nc_hint(r2 + lane, pol) : -1;
                w.nx_tag = view == 3 ? u2 : ~u2;
            } else if (r2) {
                const uintptr_t first = reinterpret_cast<uintptr_t>(r2) >> 7;
                const uintptr_t last = (reinterpret_cast<uintptr_t>(r2 + W2) - 1) >> 7;
                if (uintptr_t(lane) <= last - first)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"((first + lane) << 7));
            }
        }
        __syncwarp();
        for (int b0 = 0; b0 < W; b0 += 32) {
            const int j = b0 + lane;
            int32_t v = -1;
            if (j < W) v = have ? h0 : ld_nc_hint(row + j, pol);
            PILOT_CHECK_INDEX(w, v, view == 3 ? ix.n : ix.n_sub);
            if (view == 2 && v >= 0) v = __ldg(ix.sub2full + v);
            PILOT_CHECK_INDEX(w, v, view == 1 ? ix.n_sub : ix.n);
            uint64_t k = kKeyEmpty, worst = kKeyEmpty;
            if (view == 1 && !WIDE) {
                // stage (1): every neighbour's reduced row is copied into
                // staging slot `lane` while its visited bucket is probed, so
                // that the two round trips overlap; the rows of neighbours
                // found visited are copied but never read (reduced rows are
                // small, and kept in L2)
                w.cand()[lane] = v;
                const unsigned vb = __ballot_sync(kFull, v >= 0);
                if (vb) gather_issue_lanes(w, reinterpret_cast<const uint8_t*>(ix.red), ix.red_row_bytes, v, vb);
                const bool isnew = visit(w, v, v >= 0);
                const int m = __popc(__ballot_sync(kFull, isnew));
                n_dist += m;
                if (vb) gather_wait(w);
                if (m == 0) continue;
                const bool full = w.S == w.ef;
                worst = full ? (w.pool()[w.S - 1] & ~1ull) : kKeyEmpty;
                const uint32_t wbits = uint32_t(worst >> 32);
                // FP8 rows under L2 are always scored exactly (see the pre-filter notes)
                const bool filter = full && cfg.filter && wbits != orderable(INFINITY) && !(DT == 2 && METRIC == 0);
                bool keep = isnew;
                if (filter && isnew)
                    keep = approx_lb<DT, METRIC>(w.stage + lane * stage_stride(ix.red_row_bytes), ix.red_row_bytes,
                                                 w.qp, ix.dp_pad, DT == 2 ? ix.red_scales + v : nullptr) <=
                           from_orderable(wbits + 1u);   // nextup(worst distance)
                const unsigned kb = __ballot_sync(kFull, keep);
                if (keep) w.sel()[__popc(kb & lanemask_lt())] = lane;
                __syncwarp();
                const int m2 = __popc(kb);
                if (m2 > 0)
                    exact_staged<DT, METRIC>(w, ix.red_row_bytes, ix.red_scales, w.qp, m2,
                                             [&](int i) { return w.sel()[i]; }, 0);
                __syncwarp();
                if (keep) k = make_key(w.dist()[lane], v);
            } else {
                // the visited probe comes first: only unvisited neighbours are
                // gathered and scored
                const bool isnew = visit(w, v, v >= 0);
                const unsigned nb = __ballot_sync(kFull, isnew);
                const int m = __popc(nb);
                if (isnew) w.cand()[__popc(nb & lanemask_lt())] = v;
                __syncwarp();
                n_dist += m;
                if (m == 0) continue;
                // a full list only admits keys below its worst one: rows certified
                // above its distance are not scored exactly
                const bool full = w.S == w.ef;
                worst = full ? (w.pool()[w.S - 1] & ~1ull) : kKeyEmpty;
                const uint32_t wbits = uint32_t(worst >> 32);
                const bool filter = full && cfg.filter && wbits != orderable(INFINITY);
                const float thr = filter ? from_orderable(wbits + 1u) : INFINITY;   // nextup(worst distance)
                if (WIDE && view == 1)   // stage (1) with reduced rows too wide for 32 staging slots
                    filtered_dist<DT, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.red), ix.red_row_bytes,
                                              ix.red_scales, w.qp, m, cfg.stage_bytes, false,
                                              filter && !(DT == 2 && METRIC == 0), thr, ix.dp_pad);
                else
                    filtered_dist<0, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.full), ix.full_row_bytes, nullptr,
                                             w.q, m, cfg.stage_bytes, ix.full_host != 0, filter, thr, ix.d_pad);
                __syncwarp();
                if (lane < m) k = make_key(w.dist()[lane], w.cand()[lane]);
            }
            if (k >= worst) k = kKeyEmpty;
            const unsigned km = __ballot_sync(kFull, k != kKeyEmpty);
            const int nkeep = __popc(km);
            if (nkeep == 0) continue;
            if (nkeep <= 3) {   // a few keys: one insertion each, cheaper than sorting and merging
                for (unsigned rem = km; rem; rem &= rem - 1) insert_one(w, __shfl_sync(kFull, k, __ffs(rem) - 1), w.ef);
                continue;
            }
            k = nkeep <= 8 ? place_few(w, k, nkeep) : warp_sort32(k, lane);
            merge_new(w, k, nkeep, w.ef);
        }
        return true;
    }

    // Query rows into shared memory.
    __device__ __forceinline__ void load_query(const float* q_pad, const float* qp) {
        for (int i = w.lane; i < ix.d_pad; i += 32) w.q[i] = q_pad[i];
        for (int i = w.lane; i < ix.qp_pad; i += 32) w.qp[i] = qp[i];
        __syncwarp();
    }

    // Fast entry selection (Sec. 5) seeding stage (1) with the
    // best `ns` entries by (reduced distance, id): exact distances of the
    // scoring survivors, sorted; if the ns-th of them is not certified below
    // the bound on every other entry, an exact scan of the whole entry set
    // keeps the best ns (merged into C with ef = ns).  The clustered form
    // (use_fes = 2) routes the query to the closest coarse cluster and scans
    // only its entries the same way.  Without FES the seeds are the first ns
    // entries of the set.
    __device__ void fes(QState& st, const int32_t* fes_pos, double fes_lb) {
        const int lane = w.lane;
        int ns = cfg.fes_seeds < w.ef ? cfg.fes_seeds : w.ef;
        if (int64_t(ns) > ix.n_entry) ns = int(ix.n_entry);
        new_visited_set(w, ix.vis_stride, ix.epoch_max);
        w.S = 0;
        w.lb = 0;
        bool scan = false;
        if (cfg.use_fes == 1) {
            const int T = cfg.fes_T;
            const int32_t p = lane < T ? fes_pos[lane] : -1;
            const bool valid = p >= 0 && p < ix.n_entry;
            const unsigned vb = __ballot_sync(kFull, valid);
            const int m = __popc(vb);
            if (valid) w.cand()[__popc(vb & lanemask_lt())] = __ldg(ix.entry + p);
            __syncwarp();
            reduced_batch(m);
            __syncwarp();
            const uint64_t key = warp_sort32(lane < m ? make_key(w.dist()[lane], w.cand()[lane]) : kKeyEmpty, lane);
            const uint64_t kth = __shfl_sync(kFull, key, ns - 1);
            if (m >= ns && fes_lb >= double(nextafterf(key_dist(kth), INFINITY))) {
                if (lane < ns) w.pool()[lane] = key;
                w.S = ns;
            } else {
                scan = true;
            }
        } else if (cfg.use_fes == 0) {
            if (lane < ns) w.cand()[lane] = __ldg(ix.entry + lane);
            __syncwarp();
            reduced_batch(ns);
            __syncwarp();
            const uint64_t key = warp_sort32(lane < ns ? make_key(w.dist()[lane], w.cand()[lane]) : kKeyEmpty, lane);
            if (lane < ns) w.pool()[lane] = key;
            w.S = ns;
        }
        const int32_t* scan_list = ix.entry;   // entries scanned exactly, if any
        int64_t scan_count = ix.n_entry;
        if (cfg.use_fes == 2) {
            // clustered FES (Sec. 5): route to the closest centroid by
            // (reduced distance, cluster index), then scan that cluster
            uint64_t bestc = kKeyEmpty;
            for (int c0 = 0; c0 < ix.n_clusters; c0 += kCand) {
                const int mm = ix.n_clusters - c0 < kCand ? ix.n_clusters - c0 : kCand;
                if (lane < mm) w.cand()[lane] = c0 + lane;
                __syncwarp();
                batch_dist<0, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.centroids), ix.cent_pad * 4, nullptr,
                                      w.qp, mm, cfg.stage_bytes, false);
                __syncwarp();
                const uint64_t k = warp_min_key(lane < mm ? make_key(w.dist()[lane], w.cand()[lane]) : kKeyEmpty);
                bestc = k < bestc ? k : bestc;
                __syncwarp();
            }
            const int c = int(key_id(bestc));
            const int32_t lo = __ldg(ix.cl_offsets + c), hi = __ldg(ix.cl_offsets + c + 1);
            scan_list = ix.cl_entries + lo;
            scan_count = hi - lo;
            if (ns > hi - lo) ns = hi - lo;
            scan = true;
        }
        if (scan) {
            if (cfg.use_fes == 1) st.fallback = 1;
            const int ef_keep = w.ef;
            w.ef = ns;
            for (int64_t e0 = 0; e0 < scan_count; e0 += kCand) {
                const int mm = scan_count - e0 < kCand ? int(scan_count - e0) : kCand;
                if (lane < mm) w.cand()[lane] = __ldg(scan_list + e0 + lane);
                __syncwarp();
                reduced_batch(mm);
                __syncwarp();
                uint64_t k = lane < mm ? make_key(w.dist()[lane], w.cand()[lane]) : kKeyEmpty;
                if (w.S == w.ef && k >= w.pool()[w.S - 1]) k = kKeyEmpty;
                const int nkeep = __popc(__ballot_sync(kFull, k != kKeyEmpty));
                if (nkeep > 0) {
                    k = warp_sort32(k, lane);
                    merge_new(w, k, nkeep, ns);
                }
                __syncwarp();
            }
            w.ef = ef_keep;
        }
        __syncwarp();
        st.best = w.pool()[0];
        // stage (1) starts from the seeds, all unchecked; visited = the seeds
        visit(w, lane < w.S ? key_id(w.pool()[lane]) : 0, lane < w.S);
        w.lb = 0;
        st.phase = kStage1;
        st.it = 0;
        __syncwarp();
    }

    // Re-rank (stage (2), first part): full distances of stage (1)'s
    // candidates, a fresh visited set holding exactly their ids, C sorted.
    __device__ void rerank() {
        const int lane = w.lane;
        new_visited_set(w, ix.vis_stride, ix.epoch_max);
        for (int b0 = 0; b0 < w.S; b0 += kCand) {
            const int m = min(kCand, w.S - b0);
            int32_t orig = -1;
            if (lane < m) {
                orig = __ldg(ix.sub2full + key_id(w.pool()[b0 + lane]));
                PILOT_CHECK_INDEX(w, orig, ix.n);
                w.cand()[lane] = orig < 0 ? 0 : orig;
            }
            __syncwarp();
            full_batch(m);
            __syncwarp();
            if (lane < m) w.pool()[b0 + lane] = make_key(w.dist()[lane], orig);
            visit(w, orig, orig >= 0);
            __syncwarp();
        }
        sort_pool(w);
        w.lb = 0;
    }

    // Explicit seeds for the final stage alone (stages (1)(2) off): C starts
    // as the given distinct original ids (-1 entries skipped) with full
    // distances, all unchecked and visited, the best ef kept.
    __device__ void seed_start(QState& st, const int32_t* seeds, int count) {
        const int lane = w.lane;
        new_visited_set(w, ix.vis_stride, ix.epoch_max);
        w.S = 0;
        w.lb = 0;
        int scored = 0;
        for (int b0 = 0; b0 < count; b0 += kCand) {
            const int j = b0 + lane;
            const int32_t v = j < count ? seeds[j] : -1;
            const unsigned vb = __ballot_sync(kFull, v >= 0);
            const int m = __popc(vb);
            if (m == 0) continue;
            if (v >= 0) w.cand()[__popc(vb & lanemask_lt())] = v;
            __syncwarp();
            full_batch(m);
            __syncwarp();
            uint64_t k = kKeyEmpty;
            if (lane < m) k = make_key(w.dist()[lane], w.cand()[lane]);
            visit(w, lane < m ? w.cand()[lane] : 0, lane < m);
            scored += m;
            k = warp_sort32(k, lane);
            merge_new(w, k, m, w.ef);
            __syncwarp();
        }
        st.n_rerank = scored;
        st.best = kKeyEmpty;
        st.phase = kStage3;
        st.it = 0;
        w.lb = 0;
        __syncwarp();
    }

    // Run the staged search from its current phase for at most `budget`
    // expansions (Sec. 4.1 stages (1)-(3); Algorithm 1 in each).
    __device__ void advance(QState& st, int budget) {
        while (!w.failed && st.phase != kDone) {
            if (st.phase == kStage1) {
                if (!cfg.stage1 || !expand(1, st.e1, st.d1)) {
                    st.n_rerank = w.S;
                    st.phase = kRerank;
                } else {
                    if (++st.it >= kMaxExpansionsPerStage) {
                        st.capped = 1;
                        st.n_rerank = w.S;
                        st.phase = kRerank;
                    }
                    if (--budget <= 0) break;
                }
            } else if (st.phase == kRerank) {
                rerank();
                st.phase = kStage2;
                st.it = 0;
            } else if (st.phase == kStage2) {
                if (st.it >= cfg.stage2_expansions || !expand(2, st.e2, st.d2)) {
                    if (cfg.stage3) {   // stage (3): every candidate unchecked on the full graph
                        for (int i = w.lane; i < w.S; i += 32) w.pool()[i] &= ~1ull;
                        w.lb = 0;
                        __syncwarp();
                        st.phase = kStage3;
                    } else {
                        st.phase = kDone;
                    }
                    st.it = 0;
                } else {
                    ++st.it;
                    if (--budget <= 0) break;
                }
            } else {   // kStage3
                if (!expand(3, st.e3, st.d3)) {
                    st.phase = kDone;
                } else {
                    if (++st.it >= kMaxExpansionsPerStage) {
                        st.capped = 1;
                        st.phase = kDone;
                    }
                    if (--budget <= 0) break;
                }
            }
        }
    }

    // The first k candidates by (distance, id), padded with -1 / +inf.
    __device__ void write_output(const QState& st, int k, int32_t* ids, float* dists, int32_t* counters) {
        for (int j = w.lane; j < k; j += 32) {
            const bool ok = j < w.S && !w.failed;
            const uint64_t kk = ok ? w.pool()[j] : kKeyEmpty;
            ids[j] = ok ? key_id(kk) : -1;
            dists[j] = ok ? key_dist(kk) : INFINITY;
        }
        if (w.lane == 0 && counters) {
            counters[0] = st.e1; counters[1] = st.d1; counters[2] = st.e2; counters[3] = st.d2;
            counters[4] = st.e3; counters[5] = st.d3; counters[6] = st.n_rerank;
            counters[7] = st.best == kKeyEmpty ? -1 : __ldg(ix.sub2full + key_id(st.best));
        }
    }

    __device__ void run(int64_t q, const SearchIO& io) {
        load_query(io.q_pad + q * ix.d_pad, io.qp + q * ix.qp_pad);
        QState st{};
        w.ef = cfg.ef;
        if (io.seed_ids) seed_start(st, io.seed_ids + q * io.seed_count, io.seed_count);
        else fes(st, io.fes_pos + q * cfg.fes_T, io.fes_lb[q]);
        advance(st, 0x7FFFFFFF);
        write_output(st, cfg.k, io.out_ids + q * cfg.k, io.out_dists + q * cfg.k,
                     io.counters ? io.counters + q * 8 : nullptr);
        if (w.lane == 0) {
            if (st.fallback) atomicAdd(&io.status[3], 1);
            if (st.capped) atomicAdd(&io.status[4], 1);
        }
        __syncwarp();
    }
};

// Carve this warp's slice of shared memory and initialise its barrier.
__device__ __forceinline__ Warp setup_warp(const Layout& L, uint8_t* smem, const DevIndex& ix,
                                           const SearchConfig& cfg) {
    const int warp = threadIdx.x >> 5;
    uint8_t* base = smem + size_t(warp) * L.per_warp;
    Warp w;
    w.base = base;
    w.nx_tag = INT_MIN;
    w.nx_v0 = -1;
    w.q = reinterpret_cast<float*>(base + L.off_q);
    w.qp = reinterpret_cast<float*>(base + L.off_qp);
    w.stage = base + L.off_stage;
    w.phase = 0;
    w.red_base = reinterpret_cast<const uint8_t*>(ix.red);
    w.failed = false;
    w.lane = threadIdx.x & 31;
    w.S = 0;
    w.lb = 0;
    w.ef = 0;
    w.epoch = 0;
    w.epoch_ctr = 0;
    w.vis = nullptr;
    w.vis_mask = cfg.vis_mask;
    w.vis_qbits = cfg.vis_qbits;
    w.id_bits = ix.id_bits;
    w.overflow = 0;
    if (w.lane == 0) mbar_init(w.bar(), 1);
    __syncwarp();
    return w;
}

template <int DT, int METRIC, bool WIDE>
__global__ void __launch_bounds__(256, 2) search_kernel(DevIndex ix, SearchConfig cfg, SearchIO io, Layout L) {
    extern __shared__ __align__(128) uint8_t smem[];
    Warp w = setup_warp(L, smem, ix, cfg);
#ifdef PILOT_CHECKED
    w.status = io.status;
#endif
    const int slot = blockIdx.x * cfg.warps_per_block + (threadIdx.x >> 5);   // < ix.vis_slots (launch bound)
    w.vis = ix.vis + int64_t(slot) * ix.vis_stride;
    w.epoch_ctr = ix.vis_epoch[slot];
    Searcher<DT, METRIC, WIDE> s{ix, cfg, w};
    for (;;) {
        int64_t q = 0;
        if (w.lane == 0) q = atomicAdd(&io.status[1], 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= io.nq) break;
        if (io.bad_query[q]) {
            for (int j = w.lane; j < cfg.k; j += 32) {
                io.out_ids[q * cfg.k + j] = -1;
                io.out_dists[q * cfg.k + j] = INFINITY;
            }
            continue;
        }
        s.run(q, io);
        if (w.failed) {   // a gather timed out: report and stop taking queries
            if (w.lane == 0) atomicAdd(&io.status[2], 1);
            break;
        }
    }
    const unsigned ov = __reduce_add_sync(kFull, unsigned(w.overflow));
    if (w.lane == 0) {
        ix.vis_epoch[slot] = w.epoch_ctr;
        if (ov) atomicAdd(&io.status[7], int(ov));
    }
}

// One serving step: every active request advances by at most sio.budget
// expansions.  A request admitted in this step starts with FES (its
// projection and FES scores were computed for the step's new rows); others
// resume from their slot, and slots already finished are skipped.  Finished
// requests write their top-k to the host-mapped result rows, mark their slot
// done and raise their done flag.
template <int DT, int METRIC, bool WIDE>
__global__ void __launch_bounds__(256, 2) serve_step_kernel(DevIndex ix, SearchConfig cfg, ServeIO sio, Layout L) {
    extern __shared__ __align__(128) uint8_t smem[];
    Warp w = setup_warp(L, smem, ix, cfg);
#ifdef PILOT_CHECKED
    w.status = nullptr;
#endif
    Searcher<DT, METRIC, WIDE> s{ix, cfg, w};
    const int n_active = *reinterpret_cast<const volatile int32_t*>(sio.n_active);
    for (;;) {
        int i = 0;
        if (w.lane == 0) i = atomicAdd(sio.next, 1);
        i = __shfl_sync(kFull, i, 0);
        if (i >= n_active) break;
        const ServeEntry e = sio.entries[i];
        SlotState* ss = sio.state + e.slot;
        uint64_t* gpool = sio.pool + int64_t(e.slot) * sio.pool_stride;
        float* sq = sio.q_pad + int64_t(e.slot) * ix.d_pad;
        float* sqp = sio.qp + int64_t(e.slot) * ix.qp_pad;
        w.vis = sio.vis + int64_t(e.slot) * ix.vis_stride;
        w.failed = false;
        QState st{};
        int k;
        if (e.new_idx >= 0) {
            const float* nq = sio.new_q_pad + int64_t(e.new_idx) * ix.d_pad;
            const float* nqp = sio.new_qp + int64_t(e.new_idx) * ix.qp_pad;
            for (int j = w.lane; j < ix.d_pad; j += 32) sq[j] = nq[j];
            for (int j = w.lane; j < ix.qp_pad; j += 32) sqp[j] = nqp[j];
            s.load_query(nq, nqp);
            w.epoch_ctr = ss->epoch_ctr;
            w.ef = e.ef;
            k = e.k;
            const VisSize vs = vis_size_for(e.ef, ix.R > ix.R_sub ? ix.R : ix.R_sub, ix.id_bits, ix.vis_stride);
            w.vis_mask = vs.mask;
            w.vis_qbits = vs.qbits;
            s.fes(st, sio.new_fes_pos + int64_t(e.new_idx) * cfg.fes_T, sio.new_fes_lb[e.new_idx]);
        } else {
            // a request that finished in the previous step is listed again
            // when the host prepared this step before seeing it finish
            if (ss->phase == kDone) continue;
            s.load_query(sq, sqp);
            st.phase = ss->phase; st.it = ss->it;
            st.e1 = ss->e1; st.d1 = ss->d1; st.e2 = ss->e2; st.d2 = ss->d2; st.e3 = ss->e3; st.d3 = ss->d3;
            st.n_rerank = ss->n_rerank; st.fallback = ss->fallback; st.capped = ss->capped; st.best = ss->best;
            w.S = ss->S;
            w.lb = ss->lb;
            w.ef = ss->ef;
            w.epoch_ctr = ss->epoch_ctr;
            w.epoch = ss->epoch;
            k = ss->k;
            const VisSize vs = vis_size_for(w.ef, ix.R > ix.R_sub ? ix.R : ix.R_sub, ix.id_bits, ix.vis_stride);
            w.vis_mask = vs.mask;
            w.vis_qbits = vs.qbits;
            for (int j = w.lane; j < w.S; j += 32) w.pool()[j] = gpool[j];
            __syncwarp();
        }
        s.advance(st, sio.budget);
        if (st.phase == kDone || w.failed) {
            s.write_output(st, k, sio.res_ids + int64_t(e.slot) * sio.k_max,
                           sio.res_dists + int64_t(e.slot) * sio.k_max, sio.res_counters + int64_t(e.slot) * 8);
            __syncwarp();
            __threadfence_system();
            if (w.lane == 0) {
                ss->epoch_ctr = w.epoch_ctr;
                ss->phase = kDone;
                sio.res_done[e.slot] = w.failed ? 2 : 1;
            }
        } else {
            for (int j = w.lane; j < w.S; j += 32) gpool[j] = w.pool()[j];
            if (w.lane == 0) {
                ss->phase = st.phase; ss->it = st.it;
                ss->e1 = st.e1; ss->d1 = st.d1; ss->e2 = st.e2; ss->d2 = st.d2; ss->e3 = st.e3; ss->d3 = st.d3;
                ss->n_rerank = st.n_rerank; ss->fallback = st.fallback; ss->capped = st.capped; ss->best = st.best;
                ss->S = w.S; ss->lb = w.lb; ss->ef = w.ef; ss->k = k;
                ss->epoch_ctr = w.epoch_ctr; ss->epoch = w.epoch;
            }
        }
        __syncwarp();
    }
    const unsigned ov = __reduce_add_sync(kFull, unsigned(w.overflow));
    if (w.lane == 0 && ov && sio.vis_overflow) atomicAdd(sio.vis_overflow, int(ov));
}

template <int DT, int METRIC, bool WIDE>
cudaError_t launch_k(const DevIndex& ix, const SearchConfig& cfg_in, const SearchIO& io, cudaStream_t st,
                     int num_sms) {
    const SearchConfig& cfg = cfg_in;
    const Layout L = make_layout(ix, cfg);
    const size_t smem = size_t(L.per_warp) * cfg.warps_per_block;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > size_t(smem_max)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(search_kernel<DT, METRIC, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<DT, METRIC, WIDE>, cfg.warps_per_block * 32,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t blocks = int64_t(per_sm) * num_sms;
    if (blocks * cfg.warps_per_block > ix.vis_slots) blocks = ix.vis_slots / cfg.warps_per_block;
    const int64_t need = (io.nq + cfg.warps_per_block - 1) / cfg.warps_per_block;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaSuccess;
    search_kernel<DT, METRIC, WIDE><<<unsigned(blocks), cfg.warps_per_block * 32, smem, st>>>(ix, cfg, io, L);
    return cudaGetLastError();
}

template <int DT, int METRIC, bool WIDE>
cudaError_t serve_prepare_k(const DevIndex& ix, const SearchConfig& cfg, int num_sms, int max_warps, int* blocks,
                            size_t* smem_out) {
    const Layout L = make_layout(ix, cfg);
    const size_t smem = size_t(L.per_warp) * cfg.warps_per_block;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > size_t(smem_max)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(serve_step_kernel<DT, METRIC, WIDE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_step_kernel<DT, METRIC, WIDE>,
                                                      cfg.warps_per_block * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t b = int64_t(per_sm) * num_sms;
    const int64_t need = (max_warps + cfg.warps_per_block - 1) / cfg.warps_per_block;
    *blocks = int(b > need ? need : b);
    *smem_out = smem;
    return cudaSuccess;
}

template <int DT, int METRIC, bool WIDE>
cudaError_t serve_launch_k(const DevIndex& ix, const SearchConfig& cfg_in, const ServeIO& sio, cudaStream_t st,
                           int blocks, size_t smem) {
    const SearchConfig& cfg = cfg_in;
    serve_step_kernel<DT, METRIC, WIDE><<<unsigned(blocks), cfg.warps_per_block * 32, smem, st>>>(ix, cfg, sio,
                                                                                           make_layout(ix, cfg));
    return cudaGetLastError();
}

// Whether a configuration's reduced rows are too wide for stage (1)'s 32
// staging slots (the kernel instance without the overlapped copies).
__host__ __device__ inline bool wide_reduced(const DevIndex& ix, const SearchConfig& cfg) {
    return 32 * stage_stride(ix.red_row_bytes) > cfg.stage_bytes;
}

template <int DT, int METRIC>
cudaError_t launch_t(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st, int num_sms) {
    return wide_reduced(ix, cfg) ? launch_k<DT, METRIC, true>(ix, cfg, io, st, num_sms)
                                 : launch_k<DT, METRIC, false>(ix, cfg, io, st, num_sms);
}

template <int DT, int METRIC>
cudaError_t serve_prepare_t(const DevIndex& ix, const SearchConfig& cfg, int num_sms, int max_warps, int* blocks,
                            size_t* smem_out) {
    return wide_reduced(ix, cfg) ? serve_prepare_k<DT, METRIC, true>(ix, cfg, num_sms, max_warps, blocks, smem_out)
                                 : serve_prepare_k<DT, METRIC, false>(ix, cfg, num_sms, max_warps, blocks, smem_out);
}

template <int DT, int METRIC>
cudaError_t serve_launch_t(const DevIndex& ix, const SearchConfig& cfg, const ServeIO& sio, cudaStream_t st,
                           int blocks, size_t smem) {
    return wide_reduced(ix, cfg) ? serve_launch_k<DT, METRIC, true>(ix, cfg, sio, st, blocks, smem)
                                 : serve_launch_k<DT, METRIC, false>(ix, cfg, sio, st, blocks, smem);
}

}  // namespace

// Entry points of one reduced-row type DT (defined in search_<type>.cu).
#define PILOT_SEARCH_DT_ENTRIES(DT)                                                                          \
    cudaError_t launch_search_dt##DT(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io,       \
                                     cudaStream_t st, int num_sms);                                          \
    cudaError_t prepare_serve_step_dt##DT(const DevIndex& ix, const SearchConfig& cfg, int num_sms,         \
                                          int max_warps, int* blocks, size_t* smem);                         \
    cudaError_t launch_serve_step_dt##DT(const DevIndex& ix, const SearchConfig& cfg, const ServeIO& sio,   \
                                         cudaStream_t st, int blocks, size_t smem);
PILOT_SEARCH_DT_ENTRIES(0)
PILOT_SEARCH_DT_ENTRIES(1)
PILOT_SEARCH_DT_ENTRIES(2)
#undef PILOT_SEARCH_DT_ENTRIES

}  // namespace pilot
