/*
 * pilot.h -- C ABI of libpilot, a B300 (sm_103a) implementation of the GPU
 * search stages of PilotANN (Gui et al., arxiv 2503.21206).
 *
 * A search runs, for every query, the staged method of Sec. 4.1:
 *   project   q' = q V[:, :d']                        (Sec. 4.1 (1), SVD)
 *   FES       entry = argmin_e dist(q', e')           (Sec. 5, dense form of Table 2)
 *   stage (1) Algorithm 1 on the sampled subgraph with reduced vectors
 *   stage (2) full-vector re-rank of stage (1)'s candidates, then a fixed
 *             number (default 2) of subgraph expansions with full vectors
 *   stage (3) Algorithm 1 on the full graph with full vectors, seeded by
 *             stage (2)'s candidates and visited table (Sec. 4.1 (3))
 * and returns the first k candidates by (distance, id).
 *
 * Numerics: each distance (squared L2, or -<q,x> for inner product) and each
 * projected query component is the FP32 rounding of its exact value, the
 * paper's FP32 precision (Sec. 6.1); ties are broken by the smaller node id.
 *
 * Conventions shared by every entry point:
 *  - Every call returns a pilot_status; nothing aborts or prints.  On error
 *    pilot_last_error() returns a message for the calling thread.
 *  - Node ids are int32 original (full-graph) ids, 0 <= id < n < 2^31.
 *  - All arrays are dense, row-major, little-endian.
 */
#ifndef PILOT_H
#define PILOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pilot_index pilot_index;    /* opaque, owned by the library */
typedef struct pilot_server pilot_server;  /* opaque, owned by the library */

typedef enum {
    PILOT_OK = 0,
    PILOT_EINVAL = 1,    /* an argument is out of range or malformed */
    PILOT_ENOMEM = 2,    /* a device or pinned host allocation failed */
    PILOT_ECUDA = 3,     /* a CUDA runtime call failed */
    PILOT_EIO = 4,       /* a file could not be opened or read */
    PILOT_ETIMEOUT = 5,  /* a bounded wait ran out */
    PILOT_EBUSY = 6,     /* no capacity now (serving admission) */
    PILOT_EFORMAT = 7    /* an index file has a bad header, size or checksum */
} pilot_status;

enum { PILOT_METRIC_L2 = 0, PILOT_METRIC_IP = 1 };
enum { PILOT_REDUCED_F32 = 0, PILOT_REDUCED_BF16 = 1, PILOT_REDUCED_FP8_E4M3 = 2 };

/* Largest candidate-list size ef a search accepts. */
#define PILOT_MAX_EF 512
/* Largest graph / subgraph out-degree. */
#define PILOT_MAX_DEGREE 64

/*
 * Index description (Sec. 3, Fig. 2 (a)-(c); Sec. 4.3).  All pointers are
 * HOST pointers, except full_vecs, which may also be a DEVICE pointer of the
 * current device (the library tells them apart; a base set generated on the
 * GPU then never needs a host copy besides the library's own).
 * pilot_index_load copies everything into library-owned memory, so the caller
 * may free them as soon as the call returns.
 *
 *  graph           n x R int32, full graph, -1 padded
 *  subgraph_mask   n uint8, 1 = node kept by subgraph sampling
 *  subgraph        n x R_sub int32 in the full id space (Sec. 4.3): rows of
 *                  unsampled nodes hold only -1; every listed id is sampled
 *  svd_basis       d x dp float64, column c = right singular vector c
 *                  (Sec. 4.1 (1), X = U S V^T); the leading dp columns
 *  reduced_vecs    n_sub x dp reduced rows x V[:, :dp] of the sampled nodes in
 *                  ascending original-id order; float32, bf16 bits (uint16) or
 *                  FP8 E4M3 "fn" codes (uint8) as given by reduced_dtype
 *  reduced_scales  n_sub float32 per-row scales (FP8 only, else NULL):
 *                  value = decode(code) * scale
 *  full_vecs       n x d float32 original vectors
 *  entry_ids       n_entry int32 FES entry set, each a sampled node
 *  full_vecs_location
 *                  where the library keeps its copy of the full vectors:
 *                  PILOT_FULL_VECS_DEVICE (0, the default) in device memory,
 *                  or PILOT_FULL_VECS_HOST (1) in pinned host memory mapped
 *                  into the device's address space, for indexes whose full
 *                  vectors do not fit beside the rest (the memory-bounded
 *                  form: the GPU holds the subgraph, the reduced rows and the
 *                  entries, and the re-rank and stages (2)(3) read full rows
 *                  over the host link).  Results are identical either way.
 *  n_clusters, entry_cluster, cluster_centroids
 *                  optional coarse clusters of the entry set for the clustered
 *                  FES of Sec. 5 (use_fes = 2): entry_cluster[n_entry] int32
 *                  in [0, n_clusters), every cluster non-empty;
 *                  cluster_centroids n_clusters x dp float32 in the reduced
 *                  space.  n_clusters = 0 (and NULL arrays) when absent.
 *
 * Rejected with PILOT_EINVAL: sizes out of range (n >= 2^31, R or R_sub above
 * PILOT_MAX_DEGREE, dp > d, n_entry < 1), an id outside [-1, n), a repeated id
 * within a row, a subgraph edge to an unsampled node, an entry that is not
 * sampled, a non-finite vector or basis value.
 */
typedef struct {
    int64_t n, d, dp, R, R_sub, n_entry;
    int32_t metric;                 /* PILOT_METRIC_* */
    int32_t reduced_dtype;          /* PILOT_REDUCED_* */
    const int32_t* graph;
    const uint8_t* subgraph_mask;
    const int32_t* subgraph;
    const double* svd_basis;
    const void* reduced_vecs;
    const float* reduced_scales;
    const float* full_vecs;
    const int32_t* entry_ids;
    int32_t full_vecs_location;     /* PILOT_FULL_VECS_* (0 = device) */
    int64_t n_clusters;             /* entry clusters for the clustered FES, or 0 */
    const int32_t* entry_cluster;
    const float* cluster_centroids;
} pilot_index_desc;

#define PILOT_FULL_VECS_DEVICE 0
#define PILOT_FULL_VECS_HOST 1
/* pilot_index_load_files flag: keep the full vectors in pinned host memory */
#define PILOT_LOAD_FULL_VECS_HOST 1

/*
 * Copy an index to the current CUDA device.  *out receives the handle.  Besides
 * the arrays, the index holds the searches' visited sets: one hash table per
 * resident search warp (16 per SM) of 2 x pow2(1.25 x PILOT_MAX_EF x max(R,
 * R_sub)) bytes (16-bit words, 15 entries per 16), e.g. 64 KB per warp and
 * 155 MB in all at degree 32 on a 148-SM GPU, whatever n is below 2^24 (from
 * there on each table takes at least 2^(bits of n-1 - 8) bytes).  A search
 * with list size ef uses pow2(1.25 x max(ef, 32) x max(R, R_sub)) words of it
 * (at least 4096).  Each set carries a 12-bit epoch tag in the bucket headers,
 * so a new one costs nothing until the epochs run out (4095 sets) and the
 * table is cleared; the environment variable PILOT_VISITED_EPOCH_CYCLE=<c>,
 * read here, shortens that cycle to c sets (a testing aid: it only clears
 * more often).
 */
pilot_status pilot_index_load(const pilot_index_desc* desc, pilot_index** out);

/*
 * Load an index directory written by the offline builder: "pilot_index.txt"
 * (first line "pilot-index 1", then "key value" lines and one
 * "array <name> <i32|u8|u16|f32|f64> <bytes> <checksum hex>" line per array)
 * plus "<name>.bin" raw files.  The checksum is sum_i w_i * (2i + 1) mod 2^64
 * over the file's bytes as zero-padded little-endian 64-bit words w_i.
 * Optional: "n_clusters <r>" with arrays entry_cluster (i32, n_entry) and
 * cluster_centroids (f32, r x dp) for the clustered FES.
 * flags: 0 or PILOT_LOAD_FULL_VECS_HOST (full vectors in pinned host memory,
 * as full_vecs_location = PILOT_FULL_VECS_HOST); PILOT_EINVAL for other
 * bits.  PILOT_EIO if a file is missing, PILOT_EFORMAT on a bad
 * header, size or checksum; then the same validation as pilot_index_load.
 */
pilot_status pilot_index_load_files(const char* dir, int flags, pilot_index** out);

/* Release an index and its device memory.  NULL is ignored. */
void pilot_index_free(pilot_index* index);

/* Sizes of a loaded index (any pointer may be NULL). */
pilot_status pilot_index_info(const pilot_index* index, int64_t* n, int64_t* d, int64_t* dp, int64_t* n_sub,
                              int64_t* device_bytes);

/*
 * Search options.  Zero-initialise, then set what differs from the paper's
 * defaults: pilot_search_options_default() fills them in.
 */
typedef struct {
    int32_t stage1;             /* 1: run stage (1) (default 1) */
    int32_t stage2_expansions;  /* stage (2) subgraph expansions (default 2, Sec. 4.1 (2)) */
    int32_t stage3;             /* 1: run stage (3) (default 1) */
    int32_t use_fes;            /* 1: dense FES over the entry set (default); 2: clustered FES
                                   (Sec. 5): the query is routed to the cluster whose centroid
                                   is closest by (reduced distance, cluster index) and only
                                   that cluster's entries are scored (PILOT_EINVAL if the index
                                   has no clusters); 0: the first entries of entry_ids */
    int32_t warps_per_block;    /* search warps (one query each) per block, 1..8; 0 = automatic
                                   (the autotuned shape of the ef class, else 2) */
    int32_t stage_rows;         /* rows of the widest kind gathered per pass into shared memory, 4..32
                                   (clamped; a multiple of 4); 0 = automatic (autotuned or default) */
    int32_t* counters;          /* optional nq x 8 int32 (host or device): per query the
                                   expansions and distances of stages (1), (2), (3), the
                                   number of re-ranked candidates and the entry id */
    float* kernel_ms;           /* optional HOST array of 3 floats: device time in ms of the
                                   projection, FES scoring and search kernels of this call,
                                   from CUDA events recorded on the call's stream */
    int32_t* status_words;      /* optional HOST array of 8 int32: [3] = queries whose FES
                                   survivors were not certified (the entry set was scanned
                                   exactly), [0] = non-finite queries, [7] = visited-table
                                   insertions that found no room within 32 buckets (such a
                                   node is scored again if met again: results unchanged, the
                                   distance counters can exceed the oracle's); others reserved */
    int32_t fes_seeds;          /* entries seeding stage (1)'s candidate list: the best
                                   fes_seeds of the entry set by (reduced distance, id) with
                                   FES, the first fes_seeds entries without it; capped at ef
                                   and the entry count (default 1 = the paper's single entry;
                                   1..16, PILOT_EINVAL otherwise; 0 reads as 1) */
    const int32_t* seed_ids;    /* optional HOST array nq x seed_count of original ids that
                                   replace FES and seed the final stage alone (the experiment
                                   of Sec. 4.2: tau known neighbours plus random nodes):
                                   requires stage1 = 0, stage2_expansions = 0, stage3 = 1;
                                   C starts as the row's ids with full distances, all
                                   unchecked and visited; -1 entries are skipped; ids must be
                                   < n and distinct within a row (PILOT_EINVAL otherwise).
                                   Counters: [6] = seeds scored, [7] = -1 */
    int32_t seed_count;         /* entries per row of seed_ids, 1..ef */
    int32_t visited_entries;    /* 16-bit words of the visited table this call uses per warp:
                                   0 = automatic (pow2(1.25 x max(ef, 32) x max(R, R_sub)), at
                                   least 4096), else a cap, a power of two from
                                   max(256, 2^(bits of n-1 - 9)) to the index's table
                                   (PILOT_EINVAL otherwise).  A smaller table trades L2 reuse for
                                   insertions that find no room (status word [7]); results do
                                   not change */
} pilot_search_options;

void pilot_search_options_default(pilot_search_options* opt);

/*
 * Top-k search of nq queries (Sec. 4.1).
 *  queries    nq x d float32, host or device pointer
 *  out_ids    nq x k int32 original ids, -1 where fewer than k were found
 *  out_dists  nq x k float32 distances, +inf where fewer than k were found
 *  stream     a cudaStream_t, or NULL for the default stream
 * Host and device pointers may be mixed; the library tells them apart.  The
 * call is synchronous: when it returns the results are written.
 * PILOT_EINVAL if k < 1, ef < k, ef > PILOT_MAX_EF, nq < 0, or a query holds a
 * NaN or infinity (the other queries' results are still written).
 */
pilot_status pilot_search(pilot_index* index, const float* queries, int64_t nq, int k, int ef, int32_t* out_ids,
                          float* out_dists, void* stream);

/* pilot_search with explicit options (NULL = defaults). */
pilot_status pilot_search_ex(pilot_index* index, const float* queries, int64_t nq, int k, int ef,
                             int32_t* out_ids, float* out_dists, void* stream, const pilot_search_options* opt);

/*
 * pilot_search for callers that cannot allocate device memory during a call
 * (code that must leave every allocation to its own pool or allocator, or
 * loops that cannot afford the synchronisation an allocation brings).  The
 * paper has no counterpart; this is a library convenience.
 *
 * Same search, defaults and results as pilot_search, but the per-call scratch
 * lives in one fixed device array of PILOT_NOALLOC_SCRATCH_BYTES that the
 * library holds on every GPU it is loaded on until the process exits; the call
 * makes no cudaMalloc / cudaFree.  queries, out_ids and out_dists must be
 * DEVICE pointers (PILOT_EINVAL otherwise), and the index must already be
 * loaded.  A batch whose scratch would not fit is rejected with PILOT_EINVAL
 * and a message giving the size; split it.  The first call on a device looks
 * up the array's device address, so make that first call before capturing any
 * stream.  Every call on a device shares the array: calls whose GPU work
 * overlaps race on it.  Synchronous on `stream`, like pilot_search.
 */
#define PILOT_NOALLOC_SCRATCH_BYTES (16u << 20)
pilot_status pilot_search_noalloc(pilot_index* index, const float* queries, int64_t nq, int k, int ef,
                                  int32_t* out_ids, float* out_dists, void* stream);

/*
 * Serving (continuous batching).  A server owns device state for `slots`
 * requests in flight and drives `streams` lanes from a background thread.
 * Each lane is a CUDA stream with its own sequence of steps: a step admits
 * queued requests into free slots, then advances the lane's requests by at
 * most expansions_per_step expansions of the staged search in one persistent
 * launch replayed from a CUDA graph; a request's candidate list, visited
 * table and phase stay in device memory between steps.  A request stays on
 * its lane until it finishes, so lanes whose steps run at the same time hold
 * disjoint slots.  Requests that arrive while steps run are admitted by the
 * next idle lane and run beside them.  Each request's result equals
 * pilot_search's for the same query, k and ef.
 *
 * Admission: ef <= max_ef (the step kernel's shared memory is sized for
 * max_ef; PILOT_EINVAL above it) and k <= max_k; the number of slots is
 * max_slots or what hbm_budget_bytes holds (list, query rows and a visited
 * table of 2 x pow2(1.25 x max_ef x max(R, R_sub)) bytes per slot, independent of n
 * below 2^24 rows),
 * whichever is smaller, rounded down to a multiple of the warps the step
 * kernel keeps resident (when it holds at least one such wave); further
 * requests queue, and submit returns PILOT_EBUSY when queue_capacity
 * requests are waiting.  PILOT_EINVAL for streams outside 1..16.
 */
typedef struct {
    int32_t max_slots;            /* requests in flight at most (default 16384) */
    int32_t max_ef;               /* largest ef a request may use (default 512) */
    int32_t max_k;                /* largest k (default 100) */
    int32_t expansions_per_step;  /* per request per step (default 4096) */
    int32_t max_new_per_step;     /* admissions per step (default 8192; at most the slot count) */
    int32_t step_timeout_ms;      /* a step longer than this fails the server (default 10000) */
    int64_t queue_capacity;       /* waiting requests before PILOT_EBUSY (default 2^20) */
    int64_t hbm_budget_bytes;     /* device memory for slots; 0 = a quarter of free memory */
    int32_t streams;              /* lanes: CUDA streams with their own step sequences (1..16,
                                     default 4; 0 reads as 4) */
} pilot_serve_config;

typedef struct {
    uint64_t submitted, admitted, rejected, completed, steps;
    int32_t slots, in_flight, queued;
    int32_t visited_overflows;    /* visited-table insertions that found no room (results unchanged) */
    double qps;                   /* completed / (last completion - first submission) */
    double p50_ms, p99_ms, mean_ms;   /* submit-to-completion latency */
} pilot_serve_statistics;

void pilot_serve_config_default(pilot_serve_config* config);
/* Start a server on a loaded index (the index must outlive it). */
pilot_status pilot_serve_create(pilot_index* index, const pilot_serve_config* config, pilot_server** out);
/* Queue one query (d floats, host memory, copied); *ticket identifies it.
 * PILOT_EINVAL for k / ef outside the admission limits or a non-finite
 * value; PILOT_EBUSY when the queue is full. */
pilot_status pilot_serve_submit(pilot_server* server, const float* query, int k, int ef, uint64_t* ticket);
/* Queue n queries at once (n x d floats, host memory, copied) with their own
 * k[i] and ef[i] (host arrays); tickets[i] receives each ticket.  All or
 * nothing: PILOT_EINVAL if any request is outside the admission limits or
 * holds a non-finite value, PILOT_EBUSY if the queue cannot take all n; then
 * nothing is queued. */
pilot_status pilot_serve_submit_batch(pilot_server* server, const float* queries, int64_t n, const int32_t* k,
                                      const int32_t* ef, uint64_t* tickets);
/* Wait up to timeout_ms for a ticket; on success write k ids and distances
 * (host memory).  PILOT_ETIMEOUT if not done in time (the ticket stays
 * valid); each finished ticket can be collected once. */
pilot_status pilot_serve_wait(pilot_server* server, uint64_t ticket, int timeout_ms, int32_t* ids, float* dists);
/* pilot_serve_wait that also writes the request's 8 counters (host memory,
 * may be NULL): the same per-stage expansions and distances, re-ranked count
 * and entry id as pilot_search_options.counters. */
pilot_status pilot_serve_wait_ex(pilot_server* server, uint64_t ticket, int timeout_ms, int32_t* ids, float* dists,
                                 int32_t* counters);
pilot_status pilot_serve_stats(pilot_server* server, pilot_serve_statistics* stats);
/* Stop the background thread and free the server (pending tickets are lost). */
void pilot_serve_destroy(pilot_server* server);

/*
 * Autotuner: picks the search kernel's launch shape for one index and one
 * class of ef (the candidate list's power-of-two capacity: ef in 1..32,
 * 33..64, ..., 257..512).  The paper has no counterpart; it tunes only how
 * the same search is laid out on the GPU, so results do not change.
 *
 * Times the search kernel (CUDA events, 1 untimed + 3 timed runs each, the
 * median kept) on the caller's `queries` (nq x d float32, host or device) at
 * (k, ef), with the stage switches of `base` (stage1, stage2_expansions,
 * stage3, use_fes; NULL = the defaults; its other fields are ignored), for
 * every pair of
 *   warps_per_block  in {1, 2, 4, 8}   (queries per block; one warp each)
 *   stage_rows       in {4, 8, 12, 16, 20, 24, 32} (rows staged per gather pass)
 * whose shared memory fits, and for the defaults.  The fastest becomes the
 * index's shape for that ef class when it beats the defaults by more than 1%
 * (else the defaults stay): pilot_search / pilot_search_ex calls whose
 * options leave warps_per_block or stage_rows at 0 use it, and servers
 * created on the index afterwards whose max_ef falls in that class use its
 * stage_rows (their step kernel keeps two warps per block).
 * (pilot_search_noalloc keeps the defaults.)
 *
 * cache_path (may be NULL): a text file of lines
 *   "<key> <warps_per_block> <stage_rows> <best_ms>"
 * where key names the device model, the index shape (n, d, d', reduced
 * type, metric, R, R_sub, n_sub, entries), the ef class and the stage
 * switches.  A class holds one shape: the last tuning of it wins.  When the file
 * holds the key, its shape is applied without timing (from_cache = 1);
 * otherwise the timed result is appended.  An unreadable file counts as
 * empty; a write failure is ignored (the tuned shape still applies).
 * Errors: PILOT_EINVAL for the arguments pilot_search rejects, nq < 1 or a
 * NULL index / queries; search errors are passed on.  Not thread-safe with
 * other calls on the same index that rely on automatic shapes.
 */
typedef struct {
    int32_t warps_per_block;   /* chosen shape */
    int32_t stage_rows;
    int32_t candidates;        /* shapes timed (0 when read from the cache) */
    int32_t from_cache;        /* 1 when the shape came from cache_path */
    float best_ms;             /* median search-kernel time of the chosen shape */
    float default_ms;          /* the same for the default shape (0 from the cache) */
} pilot_tune_result;

pilot_status pilot_autotune(pilot_index* index, const float* queries, int64_t nq, int k, int ef, void* stream,
                            const pilot_search_options* base, const char* cache_path, pilot_tune_result* result);

/* The calling thread's last error message ("" if none). */
const char* pilot_last_error(void);

/* Library and ABI version, e.g. 1. */
int pilot_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PILOT_H */
