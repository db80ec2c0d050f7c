// search.cu -- the fused staged search (Sec. 4.1 stages (1)-(3), Alg. 1).
//
// A persistent kernel: every warp repeatedly takes the next query and runs,
// with all per-query state in its slice of shared memory,
//   FES check     exact distances of the FES survivors, certified against the
//                 scoring bound, else an exact scan of the entry set (Sec. 5)
//   stage (1)     Algorithm 1 on the subgraph with reduced rows (Sec. 4.1 (1))
//   re-rank       full-vector distances of stage (1)'s candidates; a fresh
//                 visited table holding exactly them (Sec. 4.1 (2))
//   stage (2)     `stage2_expansions` expansions on the subgraph with full rows
//   stage (3)     Algorithm 1 on the full graph with full rows, all candidates
//                 unchecked, reusing stage (2)'s visited table (Sec. 4.1 (3))
//   output        the first k candidates by (distance, id)
//
// Per-warp shared memory: the candidate list C (sorted 64-bit keys), the
// query and projected query, and a staging buffer for gathered rows.  The
// visited sets live in HBM: one byte per node for every warp slot, tagged with
// a per-slot epoch so that a slot is cleared only once every 255 stages.  The
// visited bytes of an expansion's neighbours are loaded together with their
// rows, so the check adds no dependent memory round trip.  Distance batches: up to 32 rows;
// eight lanes cover one 128-byte line of a row (16-byte cp.async copies into
// shared memory), each lane owns 8 rows x its chunks, and a transposing
// shuffle reduction leaves each row's sum in one lane.  New candidates are
// sorted with a warp bitonic sort and merged into C by rank.
#include <cfloat>

#include "device_common.cuh"
#include "kernels.h"

namespace pilot {
namespace {

constexpr int kCand = 32;   // distance batch (rows)
constexpr int kMaxExpansionsPerStage = 1 << 22;

struct Layout {
    int pool_cap;      // power of two >= ef
    int off_pool0, off_cand, off_dist, off_bkeys, off_q, off_qp, off_stage;
    int per_warp;
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

__host__ __device__ inline int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ __device__ inline Layout make_layout(const DevIndex& ix, const SearchConfig& cfg) {
    Layout L;
    L.pool_cap = pow2_ceil(cfg.ef < 32 ? 32 : cfg.ef);
    int o = 0;
    L.off_pool0 = o; o += L.pool_cap * 8;
    L.off_cand = o; o += kCand * 4;
    L.off_dist = o; o += kCand * 4;
    L.off_bkeys = o; o += kCand * 8;
    o = round_up(o, 16);
    L.off_q = o; o += ix.d_pad * 4;
    L.off_qp = o; o += ix.qp_pad * 4;
    o = round_up(o, 128);
    L.off_stage = o; o += cfg.stage_bytes;
    L.per_warp = round_up(o, 128);
    return L;
}

struct Warp {
    uint64_t* pool;
    uint8_t* stamps;     // this warp slot's visited bytes
    int32_t* cand;
    float* dist;
    uint64_t* bkeys;
    float* q;
    float* qp;
    uint8_t* stage;
    int S;          // candidates in C
    int lb;         // every candidate before position lb is checked
    uint32_t epoch_ctr;
    uint32_t epoch;  // 1..255: the current stage's visited tag
    int lane;
};

// Distances of rows cand[0..m) of a row array (`base`, `row_bytes` per row,
// element type DT: 0 f32, 1 bf16, 2 fp8 codes with per-row `scales`) to the
// query q held in shared memory; results in dist[0..m).
template <int DT, int METRIC>
__device__ __forceinline__ void batch_dist(Warp& w, const uint8_t* __restrict__ base, int row_bytes,
                                           const float* __restrict__ scales, const float* q, int m,
                                           int stage_bytes) {
    const int lane = w.lane;
    const int g = lane >> 3, mm = lane & 7;
    const int F8 = row_bytes >> 7;   // 16-byte chunks per lane per row
    int P = stage_bytes / row_bytes;
    P = P >= kCand ? kCand : (P & ~3);
    const int jrows = (m + 3) >> 2;   // row slots any lane needs (warp-uniform)
    DF acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = DF{0.0f, 0.0f};
    for (int r0 = 0; r0 < m; r0 += P) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = g + 4 * j;
            if (r >= r0 && r < r0 + P && r < m) {
                const uint8_t* src = base + int64_t(w.cand[r]) * row_bytes;
                uint8_t* dst = w.stage + (r - r0) * row_bytes;
                for (int t = 0; t < F8; ++t) cp_async16(dst + (mm + 8 * t) * 16, src + (mm + 8 * t) * 16);
            }
        }
        cp_async_wait_all();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = g + 4 * j;
            // every lane works on row slot j when any lane needs it (rows past m
            // hold stale data whose result is discarded), so the warp stays converged
            if (j < jrows && 4 * j >= r0 && 4 * j < r0 + P) {
                const uint8_t* srow = w.stage + (r - r0) * row_bytes;
                float sc = 1.0f;
                if (DT == 2) sc = r < m ? __ldg(scales + w.cand[r]) : 1.0f;
                for (int t = 0; t < F8; ++t) {
                    const int c = mm + 8 * t;
                    uint4 v = *reinterpret_cast<const uint4*>(srow + c * 16);
                    if (DT == 0) {
                        float4 qv = *reinterpret_cast<const float4*>(q + c * 4);
                        float x[4] = {__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                      __uint_as_float(v.w)};
                        float qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (METRIC == 0) l2_acc(acc[j], qa[e], x[e]);
                            else ip_acc(acc[j], qa[e], x[e]);
                        }
                    } else if (DT == 1) {
                        uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float2 qv = *reinterpret_cast<const float2*>(q + c * 8 + h * 2);
                            float x0 = bf16_to_f32(wv[h] & 0xFFFFu), x1 = bf16_to_f32(wv[h] >> 16);
                            if (METRIC == 0) {
                                l2_acc(acc[j], qv.x, x0);
                                l2_acc(acc[j], qv.y, x1);
                            } else {
                                ip_acc(acc[j], qv.x, x0);
                                ip_acc(acc[j], qv.y, x1);
                            }
                        }
                    } else {
                        uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float4 qv = *reinterpret_cast<const float4*>(q + c * 16 + h * 4);
                            float qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                float xl;
                                float xh = two_prod(e4m3_to_f32((wv[h] >> (8 * b)) & 0xFFu), sc, xl);
                                if (METRIC == 0) l2_acc2(acc[j], qa[b], xh, xl);
                                else ip_acc2(acc[j], qa[b], xh, xl);
                            }
                        }
                    }
                }
            }
        }
    }
    // Transposing reduction over the eight lanes of a group: afterwards lane
    // (g, mm) holds the full sum of row g + 4 * mm.
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = mm & 4;
        DF send = up ? acc[i] : acc[i + 4];
        DF keep = up ? acc[i + 4] : acc[i];
        acc[i] = df_add(keep, df_shfl_xor(send, 4));
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = mm & 2;
        DF send = up ? acc[i] : acc[i + 2];
        DF keep = up ? acc[i + 2] : acc[i];
        acc[i] = df_add(keep, df_shfl_xor(send, 2));
    }
    {
        const bool up = mm & 1;
        DF send = up ? acc[0] : acc[1];
        DF keep = up ? acc[1] : acc[0];
        acc[0] = df_add(keep, df_shfl_xor(send, 1));
    }
    const int r = g + 4 * mm;
    if (r < m) w.dist[r] = df_finish(acc[0], METRIC);
}

__device__ __forceinline__ uint64_t warp_min(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t x = __shfl_xor_sync(kFull, v, o);
        v = x < v ? x : v;
    }
    return v;
}

// Merge nb sorted new keys (lanes 0..nb-1, kKeyEmpty beyond) into C in place.
// A new key equal to one already in C (same distance and id) is dropped.  Each
// kept key lands at (its rank among the new keys) + (its lower bound in C);
// output positions are filled from the last 32-slot chunk down to the first
// changed one, every lane reading its source before any lane writes, so an
// element is always read before it is overwritten.  C keeps its ef best.
__device__ __forceinline__ void merge_new(Warp& w, uint64_t key, int nb, int ef) {
    const int lane = w.lane;
    uint64_t* A = w.pool;
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
    if (mine) w.bkeys[ci] = key;
    const int Snew = min(S + nb2, ef);
    const int lo_pos = __reduce_min_sync(kFull, np);
    __syncwarp();
    if (lo_pos >= Snew) return;
    for (int c = (Snew - 1) >> 5; c >= (lo_pos >> 5); --c) {
        const int base = c << 5;
        const int pos = base + lane;
        const unsigned bit = (mine && np >= base && np < base + 32) ? (1u << (np - base)) : 0u;
        const unsigned mask_c = __reduce_or_sync(kFull, bit);
        const int before = __popc(__ballot_sync(kFull, mine && np < base));
        const bool write = pos < Snew && pos >= lo_pos;
        uint64_t val = 0;
        if (write) {
            const unsigned upto = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
            const int kle = before + __popc(mask_c & upto);
            val = ((mask_c >> lane) & 1u) ? w.bkeys[kle - 1] : A[pos - kle];
        }
        __syncwarp();
        if (write) A[pos] = val;
        __syncwarp();
    }
    w.S = Snew;
    if (lo_pos < w.lb) w.lb = lo_pos;
}

// Ascending bitonic sort of C in place (the re-rank), padded to a power of two.
__device__ __forceinline__ void sort_pool(Warp& w, int cap) {
    uint64_t* A = w.pool;
    int N = 1;
    while (N < w.S) N <<= 1;
    for (int i = w.S + w.lane; i < N && i < cap; i += 32) A[i] = kKeyEmpty;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = w.lane; i < N; i += 32) {
                const int l = i ^ j;
                if (l > i) {
                    uint64_t a = A[i], b = A[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        A[i] = b;
                        A[l] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Start a new visited set for this warp slot.  Epochs cycle through 1..255;
// before a cycle restarts the slot's bytes are cleared.
__device__ __forceinline__ void new_visited_set(Warp& w, int64_t stride) {
    w.epoch_ctr += 1;
    const uint32_t r = w.epoch_ctr % 255u;
    if (r == 0) {
        uint4* p = reinterpret_cast<uint4*>(w.stamps);
        const int64_t n16 = stride >> 4;
        for (int64_t i = w.lane; i < n16; i += 32) p[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    w.epoch = r + 1;
    __syncwarp();
}

template <int DT, int METRIC>
struct Searcher {
    const DevIndex& ix;
    const SearchConfig& cfg;
    Warp& w;

    __device__ __forceinline__ void reduced_batch(int m) {
        batch_dist<DT, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.red), ix.red_row_bytes, ix.red_scales, w.qp,
                               m, cfg.stage_bytes);
    }
    __device__ __forceinline__ void full_batch(int m) {
        batch_dist<0, METRIC>(w, reinterpret_cast<const uint8_t*>(ix.full), ix.full_row_bytes, nullptr, w.q, m,
                              cfg.stage_bytes);
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
            const bool unc = i < w.S && !(w.pool[i] & 1ull);
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
        const uint64_t key = w.pool[idx];
        __syncwarp();
        if (lane == 0) w.pool[idx] = key | 1ull;
        w.lb = idx + 1;
        n_exp += 1;
        const int32_t u = key_id(key);
        const int32_t* row = adjacency(view, u);
        const int W = view == 3 ? ix.R : (row ? ix.R_sub : 0);
        // the next expansion most likely takes the second unchecked candidate:
        // bring its adjacency row into L2 while this one is processed
        if (idx2 >= 0 && lane == 0) {
            const int32_t* r2 = adjacency(view, key_id(w.pool[idx2]));
            if (r2) asm volatile("prefetch.global.L2 [%0];" ::"l"(r2));
        }
        __syncwarp();
        for (int b0 = 0; b0 < W; b0 += 32) {
            const int j = b0 + lane;
            int32_t v = j < W ? __ldg(row + j) : -1;
            if (view == 2 && v >= 0) v = __ldg(ix.sub2full + v);
            const unsigned vb = __ballot_sync(kFull, v >= 0);
            const int m = __popc(vb);
            if (m == 0) continue;
            if (v >= 0) w.cand[__popc(vb & lanemask_lt())] = v;
            __syncwarp();
            // visited bytes of all neighbours, in flight with their rows; the
            // distance batch covers every neighbour and the visited ones are
            // dropped afterwards
            const int32_t mine = lane < m ? w.cand[lane] : 0;
            const uint32_t tag = lane < m ? uint32_t(w.stamps[mine]) : w.epoch;
            if (view == 1) reduced_batch(m);
            else full_batch(m);
            const bool isnew = tag != w.epoch;
            if (isnew) w.stamps[mine] = uint8_t(w.epoch);
            const int cnt = __popc(__ballot_sync(kFull, isnew));
            n_dist += cnt;
            uint64_t k = isnew ? make_key(w.dist[lane], mine) : kKeyEmpty;
            // a full list only admits keys below its worst one
            if (w.S == cfg.ef && k >= (w.pool[w.S - 1] & ~1ull)) k = kKeyEmpty;
            const int nkeep = __popc(__ballot_sync(kFull, k != kKeyEmpty));
            if (nkeep == 0) continue;
            k = warp_sort32(k, lane);
            merge_new(w, k, nkeep, cfg.ef);
        }
        return true;
    }

    __device__ void run(int64_t q, const SearchIO& io, int32_t* cnt_out) {
        const int lane = w.lane;
        // query rows into shared memory
        for (int i = lane; i < ix.d_pad; i += 32) w.q[i] = io.q_pad[q * ix.d_pad + i];
        for (int i = lane; i < ix.qp_pad; i += 32) w.qp[i] = io.qp[q * ix.qp_pad + i];
        __syncwarp();
        int status_fallback = 0;

        // ---- fast entry selection: exact check of the scoring survivors
        uint64_t best;
        if (cfg.use_fes) {
            const int T = cfg.fes_T;
            const int32_t p = lane < T ? io.fes_pos[q * T + lane] : -1;
            const bool valid = p >= 0 && p < ix.n_entry;
            const unsigned vb = __ballot_sync(kFull, valid);
            const int m = __popc(vb);
            if (valid) w.cand[__popc(vb & lanemask_lt())] = __ldg(ix.entry + p);
            __syncwarp();
            reduced_batch(m);
            __syncwarp();
            best = warp_min(lane < m ? make_key(w.dist[lane], w.cand[lane]) : kKeyEmpty);
            const double lb = io.fes_lb[q];
            const float dstar = key_dist(best);
            if (!(lb >= double(nextafterf(dstar, INFINITY)))) {
                status_fallback = 1;
                best = kKeyEmpty;
                for (int64_t e0 = 0; e0 < ix.n_entry; e0 += kCand) {
                    const int mm = ix.n_entry - e0 < kCand ? int(ix.n_entry - e0) : kCand;
                    if (lane < mm) w.cand[lane] = __ldg(ix.entry + e0 + lane);
                    __syncwarp();
                    reduced_batch(mm);
                    __syncwarp();
                    const uint64_t b = warp_min(lane < mm ? make_key(w.dist[lane], w.cand[lane]) : kKeyEmpty);
                    best = b < best ? b : best;
                    __syncwarp();
                }
            }
        } else {
            if (lane == 0) w.cand[0] = __ldg(ix.entry);
            __syncwarp();
            reduced_batch(1);
            __syncwarp();
            best = make_key(w.dist[0], w.cand[0]);
        }

        // ---- stage (1): Algorithm 1 on the subgraph, reduced rows
        int e1 = 0, d1 = 0, e2 = 0, d2 = 0, e3 = 0, d3 = 0;
        new_visited_set(w, ix.stamp_stride);
        if (lane == 0) {
            w.pool[0] = best;
            w.stamps[key_id(best)] = uint8_t(w.epoch);
        }
        w.S = 1;
        w.lb = 0;
        __syncwarp();
        bool capped = false;
        if (cfg.stage1) {
            int it = 0;
            while (expand(1, e1, d1))
                if (++it >= kMaxExpansionsPerStage) { capped = true; break; }
        }
        const int n_rerank = w.S;

        // ---- re-rank: full distances, fresh visited table = ids(C)
        new_visited_set(w, ix.stamp_stride);
        for (int b0 = 0; b0 < w.S; b0 += kCand) {
            const int m = min(kCand, w.S - b0);
            int32_t orig = -1;
            if (lane < m) {
                orig = __ldg(ix.sub2full + key_id(w.pool[b0 + lane]));
                w.cand[lane] = orig;
            }
            __syncwarp();
            full_batch(m);
            __syncwarp();
            if (lane < m) {
                w.pool[b0 + lane] = make_key(w.dist[lane], orig);
                w.stamps[orig] = uint8_t(w.epoch);
            }
            __syncwarp();
        }
        sort_pool(w, 0x7FFFFFFF);
        w.lb = 0;

        // ---- stage (2): a fixed number of subgraph expansions, full rows
        for (int it = 0; it < cfg.stage2_expansions; ++it)
            if (!expand(2, e2, d2)) break;

        // ---- stage (3): Algorithm 1 on the full graph, all unchecked
        if (cfg.stage3) {
            for (int i = lane; i < w.S; i += 32) w.pool[i] &= ~1ull;
            w.lb = 0;
            __syncwarp();
            int it = 0;
            while (expand(3, e3, d3))
                if (++it >= kMaxExpansionsPerStage) { capped = true; break; }
        }

        // ---- output: first k by (distance, id)
        for (int j = lane; j < cfg.k; j += 32) {
            const bool ok = j < w.S;
            const uint64_t kk = ok ? w.pool[j] : kKeyEmpty;
            io.out_ids[q * cfg.k + j] = ok ? key_id(kk) : -1;
            io.out_dists[q * cfg.k + j] = ok ? key_dist(kk) : INFINITY;
        }
        if (lane == 0) {
            if (cnt_out) {
                int32_t* c = cnt_out + q * 8;
                c[0] = e1; c[1] = d1; c[2] = e2; c[3] = d2; c[4] = e3; c[5] = d3; c[6] = n_rerank;
                c[7] = __ldg(ix.sub2full + key_id(best));
            }
            if (status_fallback) atomicAdd(&io.status[3], 1);
            if (capped) atomicAdd(&io.status[4], 1);
        }
        __syncwarp();
    }
};

template <int DT, int METRIC>
__global__ void __launch_bounds__(256) search_kernel(DevIndex ix, SearchConfig cfg, SearchIO io, Layout L) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int warp = threadIdx.x >> 5;
    uint8_t* base = smem + size_t(warp) * L.per_warp;
    Warp w;
    w.pool = reinterpret_cast<uint64_t*>(base + L.off_pool0);
    const int slot = blockIdx.x * cfg.warps_per_block + warp;   // < ix.stamp_slots (launch bound)
    w.stamps = ix.stamps + int64_t(slot) * ix.stamp_stride;
    w.epoch_ctr = ix.stamp_epoch[slot];
    w.epoch = 0;
    w.cand = reinterpret_cast<int32_t*>(base + L.off_cand);
    w.dist = reinterpret_cast<float*>(base + L.off_dist);
    w.bkeys = reinterpret_cast<uint64_t*>(base + L.off_bkeys);
    w.q = reinterpret_cast<float*>(base + L.off_q);
    w.qp = reinterpret_cast<float*>(base + L.off_qp);
    w.stage = base + L.off_stage;
    w.lane = threadIdx.x & 31;
    w.S = 0;
    w.lb = 0;
    Searcher<DT, METRIC> s{ix, cfg, w};
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
        s.run(q, io, io.counters);
    }
    if (w.lane == 0) ix.stamp_epoch[slot] = w.epoch_ctr;
}

template <int DT, int METRIC>
cudaError_t launch_t(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st,
                     int num_sms) {
    const Layout L = make_layout(ix, cfg);
    const size_t smem = size_t(L.per_warp) * cfg.warps_per_block;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > size_t(smem_max)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(search_kernel<DT, METRIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<DT, METRIC>, cfg.warps_per_block * 32,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t blocks = int64_t(per_sm) * num_sms;
    if (blocks * cfg.warps_per_block > ix.stamp_slots) blocks = ix.stamp_slots / cfg.warps_per_block;
    const int64_t need = (io.nq + cfg.warps_per_block - 1) / cfg.warps_per_block;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaSuccess;
    search_kernel<DT, METRIC><<<unsigned(blocks), cfg.warps_per_block * 32, smem, st>>>(ix, cfg, io, L);
    return cudaGetLastError();
}

}  // namespace

size_t search_smem_per_warp(const DevIndex& ix, const SearchConfig& cfg) { return make_layout(ix, cfg).per_warp; }

SearchConfig default_search_config(const DevIndex& ix, int k, int ef) {
    SearchConfig cfg{};
    cfg.k = k;
    cfg.ef = ef;
    cfg.stage1 = 1;
    cfg.stage2_expansions = 2;
    cfg.stage3 = 1;
    cfg.use_fes = 1;
    cfg.fes_T = 8;
    cfg.warps_per_block = 2;
    int stage = 4 * (ix.full_row_bytes > ix.red_row_bytes ? ix.full_row_bytes : ix.red_row_bytes);
    const int full32 = 32 * ix.full_row_bytes < 16384 ? 32 * ix.full_row_bytes : 16384;
    stage = stage > full32 ? stage : full32;
    cfg.stage_bytes = stage > 32 * ix.red_row_bytes ? stage : 32 * ix.red_row_bytes;
    return cfg;
}

cudaError_t launch_search(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st,
                          int num_sms) {
    if (io.nq == 0) return cudaSuccess;
    const int key = ix.red_dtype * 2 + ix.metric;
    switch (key) {
        case 0: return launch_t<0, 0>(ix, cfg, io, st, num_sms);
        case 1: return launch_t<0, 1>(ix, cfg, io, st, num_sms);
        case 2: return launch_t<1, 0>(ix, cfg, io, st, num_sms);
        case 3: return launch_t<1, 1>(ix, cfg, io, st, num_sms);
        case 4: return launch_t<2, 0>(ix, cfg, io, st, num_sms);
        case 5: return launch_t<2, 1>(ix, cfg, io, st, num_sms);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pilot
