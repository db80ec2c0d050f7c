// kernels.h -- launch interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pilot {

constexpr int kFesT = 16;   // FES survivors per query

// Device-resident index (library-owned).  Rows are padded with zeros to a
// multiple of 128 bytes so that eight lanes cover one 128-byte line.
struct DevIndex {
    int64_t n, d, dp, n_sub, n_entry;
    int R, R_sub;
    int metric;          // 0 L2, 1 IP
    int red_dtype;       // 0 f32, 1 bf16, 2 fp8
    int d_pad;           // full row length in floats
    int dp_pad;          // reduced row length in elements
    int full_row_bytes;  // d_pad * 4
    int red_row_bytes;   // dp_pad * element size
    int qp_pad;          // projected-query row length in floats (multiple of 64)
    int full_host;       // 1: the full rows live in mapped pinned host memory (read with plain loads)
    const int32_t* graph;      // n x R original ids
    const int32_t* sub_adj;    // n_sub x R_sub compact ids
    const int32_t* sub2full;   // n_sub
    const int32_t* full2sub;   // n (-1 for unsampled)
    const void* red;           // n_sub x dp_pad
    const float* red_scales;   // n_sub (fp8) or null
    const float* full;         // n x d_pad
    const float2* basis;       // d x qp_pad, (hi, lo) FP32 pair of each FP64 basis value
    const int32_t* entry;      // n_entry compact ids
    const float* entry_norm2;  // ||e||^2 (FP32 of the FP64 value), +inf past n_entry to whole 256-entry tiles
    float entry_max_norm;      // max ||e||
    const uint16_t* entry_bf16;   // entries as BF16, 256-row tiles in the UMMA K-major core-matrix layout
    // clustered FES: centroid rows (n_clusters x cent_pad FP32, 128-byte rows),
    // the entries' compact ids grouped by cluster, and each cluster's range
    int n_clusters;
    int cent_pad;
    const float* centroids;
    const int32_t* cl_entries;
    const int32_t* cl_offsets;   // n_clusters + 1
    // Visited sets: one open-addressing hash table per warp slot (vis_slots
    // slots of vis_stride 16-bit words each, a power of two), in 32-byte
    // buckets of 16 words (one sector): word 0 is the bucket's header
    // (epoch << 4 | count), words 1..15 its entries.  A node is split by a
    // bijection of [0, 2^id_bits) into a bucket index and a quotient, so an
    // entry stores only the quotient and its distance from the home bucket
    // (see visit() in search_impl.cuh); a bucket whose header carries another
    // epoch is empty, so a new set costs one epoch step and a slot is cleared
    // only when its epoch counter wraps.  The size depends on ef and the
    // degree, not on n (beyond a floor of 2^(id_bits - 9) words that keeps
    // quotients within 13 bits).  vis_epoch holds each slot's running epoch
    // counter across launches.
    uint16_t* vis;
    uint32_t* vis_epoch;
    int64_t vis_stride;
    int vis_slots;
    int id_bits;         // bits of a node id: n - 1 < 2^id_bits
    uint32_t epoch_max;  // epochs per cycle: at most kVisEpochs
};

constexpr int kVisBucket = 16;       // 16-bit words per bucket (32 bytes): a header and 15 entries
constexpr int kVisMaxProbe = 7;      // buckets probed (home + 0..6) before an insertion gives up
constexpr uint32_t kVisEpochs = 4095;  // 12-bit epoch field of a bucket header
constexpr int kVisQuotientBits = 13;   // an entry is (quotient << 3) | (probe + 1)

// Words of the visited table a search with list size ef uses: the power of
// two >= 1.25 x max(ef, 32) x the larger degree, at least 4096 and at least
// 2^(id_bits - 9) (so that 2^(id_bits - 13) buckets or more leave quotients of
// at most 13 bits).  A set (stage (1), or the re-rank with stages (2) and
// (3)) visits at most (its expansions + 1) x degree nodes; measured, under
// 0.8 x ef x degree plus ef at ef >= 64, so the 15 entries of each 16 words
// stay at most about 70% full.
__host__ __device__ inline int64_t vis_entries_for(int ef, int max_degree, int id_bits) {
    int64_t want = int64_t(ef < 32 ? 32 : ef) * max_degree * 5 / 4, h = 4096;
    const int64_t floor_words = id_bits > 9 ? (int64_t(1) << (id_bits - 9)) : 1;
    if (want < floor_words) want = floor_words;
    while (h < want) h <<= 1;
    return h;
}

// Smallest table (in words) a search may be capped to on an index with
// id_bits-bit ids: 256, or the quotient floor when larger.
__host__ __device__ inline int64_t vis_min_entries(int id_bits) {
    const int64_t f = id_bits > 9 ? (int64_t(1) << (id_bits - 9)) : 1;
    return f > 256 ? f : 256;
}

// Bucket mask and quotient width of a table of vis_entries_for(ef, ...)
// words, capped at entries_per_slot (both powers of two >= vis_min_entries).
struct VisSize {
    uint32_t mask;
    int qbits;
};
__host__ __device__ inline VisSize vis_size_for(int ef, int max_degree, int id_bits, int64_t entries_per_slot) {
    int64_t h = vis_entries_for(ef, max_degree, id_bits);
    if (h > entries_per_slot) h = entries_per_slot;
    const int64_t buckets = h / kVisBucket;
    int lg = 0;
    while ((int64_t(1) << lg) < buckets) ++lg;
    const int q = id_bits - lg;
    return VisSize{uint32_t(buckets - 1), q > 0 ? q : 0};
}

struct SearchConfig {
    int k, ef;
    int stage1, stage2_expansions, stage3, use_fes;
    int warps_per_block;
    int fes_T;
    int fes_seeds;       // entries seeding stage (1) (1..kFesT)
    int stage_bytes;     // per-warp row staging buffer
    uint32_t vis_mask;   // buckets of the visited table in use - 1 (a power of two - 1)
    int vis_qbits;       // quotient bits of a visited entry: id_bits - log2(buckets), at most 13
    int filter;          // 1: certified FP32 pre-filter once the list is full
};

// Byte stride of gathered rows in a warp's staging buffer: 16 bytes more than
// the row, so that lanes reading the same chunk of different rows (one row
// per lane) fall in different shared-memory banks.
__host__ __device__ inline int stage_stride(int row_bytes) { return row_bytes + 16; }

// Per-call device buffers.
struct SearchIO {
    const float* queries;      // nq x d (caller layout)
    int64_t nq;
    float* q_pad;              // nq x d_pad
    float* qp;                 // nq x qp_pad
    uint16_t* qp_bf16;         // q' as BF16, 128-row tiles in the UMMA K-major core-matrix layout
    int32_t* fes_pos;          // nq x fes_T entry positions
    double* fes_lb;            // nq lower bound on excluded entries' distances
    int32_t* out_ids;          // nq x k
    float* out_dists;          // nq x k
    int32_t* counters;         // nq x 8 or null
    int32_t* bad_query;        // nq flags (non-finite input)
    int32_t* status;           // [0] non-finite queries, [1] next query, [2] gather timeouts,
                               // [3] FES fallbacks, [4] expansion-cap hits, [5] FES kernel timeouts,
                               // [6] out-of-range indices skipped (checked build),
                               // [7] visited insertions that found no room
    const int32_t* seed_ids;   // nq x seed_count original ids (-1 skipped) seeding the final stage, or null
    int seed_count;
};

// ------------------------------------------------------------- serving --

// One request in a serving step: its slot, and for a request admitted in
// this step its row in the step's new-request buffers (else -1).
struct ServeEntry {
    int32_t slot, new_idx, k, ef;
};

// A slot's search state, kept in device memory between steps.
struct SlotState {
    int32_t phase, it, e1, d1, e2, d2, e3, d3, n_rerank, fallback, capped;
    int32_t S, lb, ef, k, pad;
    uint32_t epoch_ctr, epoch;
    uint64_t best;
};

struct ServeIO {
    const ServeEntry* entries;   // n_active entries (host-mapped)
    const int32_t* n_active;     // host-mapped
    int32_t* next;               // device counter, zeroed before each step
    SlotState* state;            // per slot
    uint64_t* pool;              // per slot, pool_stride keys
    int pool_stride;
    float* q_pad;                // per slot, d_pad floats
    float* qp;                   // per slot, qp_pad floats
    const float* new_q_pad;      // this step's new requests (dense rows)
    const float* new_qp;
    const int32_t* new_fes_pos;
    const double* new_fes_lb;
    uint16_t* vis;               // per slot, vis_stride words of the index's layout
    int32_t* vis_overflow;       // device counter of visited insertions that found no room
    int32_t* res_ids;            // per slot, k_max (host-mapped)
    float* res_dists;            // per slot, k_max (host-mapped)
    int32_t* res_done;           // per slot: 1 done, 2 failed (host-mapped)
    int32_t* res_counters;       // per slot, 8 (host-mapped)
    int k_max;
    int budget;                  // expansions per slot per step
};

// Set the step kernel's attributes and size its grid (call outside capture).
cudaError_t prepare_serve_step(const DevIndex& ix, const SearchConfig& cfg, int num_sms, int max_warps, int* blocks,
                               size_t* smem);
// Launch one step (capturable).
cudaError_t launch_serve_step(const DevIndex& ix, const SearchConfig& cfg, const ServeIO& sio, cudaStream_t st,
                              int blocks, size_t smem);
size_t serve_smem_per_block(const DevIndex& ix, const SearchConfig& cfg);

cudaError_t launch_project(const DevIndex& ix, const SearchIO& io, cudaStream_t st);
cudaError_t launch_fes_mma(const DevIndex& ix, const SearchIO& io, cudaStream_t st);

// Element offset of (row, col) in a tile-blocked UMMA K-major operand with
// `tile_rows`-row tiles and kp columns: 8 x 8 core matrices, K-adjacent ones 64
// elements apart, 8-row groups kp * 8 elements apart.
__host__ __device__ inline int64_t umma_kmajor_offset(int64_t row, int col, int tile_rows, int kp) {
    const int64_t t = row / tile_rows;
    const int r = int(row % tile_rows);
    return t * int64_t(tile_rows) * kp + int64_t(r >> 3) * (kp * 8) + (col >> 3) * 64 + (r & 7) * 8 + (col & 7);
}
cudaError_t launch_search(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st,
                          int num_sms);
size_t search_smem_per_warp(const DevIndex& ix, const SearchConfig& cfg);
// The defaults of every search entry point (stages as in the paper, T = 8 FES
// survivors, automatic staging size).
SearchConfig default_search_config(const DevIndex& ix, int k, int ef);
// Stage `rows` rows of the widest row kind per gather pass (4..32).
void set_stage_rows(const DevIndex& ix, SearchConfig& cfg, int rows);
// Size the visited table of cfg for its ef within entries_per_slot.
void set_visited_size(const DevIndex& ix, SearchConfig& cfg, int64_t entries_per_slot);

// Internal view of a loaded index for entry points outside pilot_api.cu.
// Search shape chosen by the autotuner for one class of ef: the candidate
// list's power-of-two capacity 2^c, c = 5..9.  Zeros keep the defaults.
struct TunedShape {
    int warps_per_block;
    int stage_rows;
};
constexpr int kEfClasses = 10;
inline int ef_class(int ef) {
    int c = 5;
    while (c < kEfClasses - 1 && (1 << c) < ef) ++c;
    return c;
}

struct IndexView {
    const DevIndex* dev;
    int device;
    int num_sms;
    int32_t* status_host;   // pinned, 8 words
    void* mutex;            // std::mutex guarding per-index state
    TunedShape* tuned;      // kEfClasses entries, guarded by `mutex`
};
int search_blocks_per_sm(const DevIndex& ix, const SearchConfig& cfg);

}  // namespace pilot
