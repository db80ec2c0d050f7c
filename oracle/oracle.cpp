// oracle.cpp -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
//
// A plain, slow, single-purpose CPU restatement of the PilotANN top-k search
// (Gui et al., "PilotANN: Memory-Bounded GPU Acceleration for Vector Search",
// arxiv 2503.21206).  Only the tests, the smoke check and the benchmark's CPU
// baseline leg may load this library; the product search path never does.
//
// Arithmetic: every inner product / squared difference is accumulated in
// FP64 over the stored inputs (FP32 rows, or BF16 / FP8-E4M3 rows decoded
// exactly), and each finished distance (and each projected query component)
// is rounded ONCE to FP32, the precision the paper fixes for all distance
// calculations (Sec. 6.1, "Experimental Setup").  Every ordering decision is
// taken on those FP32 values with ties broken by the original node id.
//
// No blocking, fusion or reordering: loops follow the definitions in the
// paper's order.  Nothing here is shared with the GPU path.
//
// Parity pins (tests/test_oracle_pins.py): orthonormal basis, projection
// with d'=d equals the full distance, projected <= full distance (Sec. 4.1),
// brute-force limit (subgraph = full graph, d'=d, ef >= N), hand-computed
// Algorithm 1 traces (tests/golden/), dense FES == argmin over the entry set
// (Table 2, "FES (1 block)"), graceful degradation (Sec. 4.1 "Summary").

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- inputs --

struct Index {
    int64_t n, d, dp, R, R_sub, n_entry;
    int metric;                     // 0: squared L2, 1: inner product (-<q,x>)
    const int32_t* graph;           // n x R, original ids, -1 padded
    const uint8_t* subgraph_mask;   // n, 1 = sampled (Sec. 4.3)
    const int32_t* subgraph;        // n x R_sub, original ids, -1 padded; rows of unsampled nodes unused
    const double* basis;            // d x dp, basis[j*dp + c] = V[j][c] (right singular vectors)
    const void* reduced;            // n_sub x dp, rows of sampled nodes in ascending original id order
    int reduced_dtype;              // 0: FP32, 1: BF16, 2: FP8 E4M3 (fn) with per-row FP32 scale
    const float* reduced_scales;    // n_sub (FP8 only)
    const float* full;              // n x d FP32 original vectors
    const int32_t* entry_ids;       // n_entry original ids (all sampled)
    int64_t n_clusters;             // clustered FES (Sec. 5): coarse clusters of the entry set, or 0
    const int32_t* entry_cluster;   // n_entry cluster of each entry
    const float* centroids;         // n_clusters x dp FP32 centroids in the reduced space
};

struct Params {
    int k, ef;
    int stage1;              // 1: run stage (1) on the subgraph (Sec. 4.1)
    int stage2_expansions;   // expansions of stage (2) on the subgraph (paper: 2)
    int stage3;              // 1: run stage (3) on the full graph
    int use_fes;             // 1: dense FES over the entry set; 2: clustered FES; 0: the first entries
    int fes_seeds;           // entries seeding stage (1) (the paper: 1)
    int nthreads;
    int seed_count;          // with seed_ids: entries per query row
    const int32_t* seed_ids; // nq x seed_count original ids seeding the final stage alone, or null
};

// Per-query outputs.  Any pointer may be null.
struct Outputs {
    int32_t* ids;        // nq x k, original ids, -1 padded
    float* dists;        // nq x k, +inf padded
    int32_t* counters;   // nq x 8: exp1, dist1, exp2, dist2, exp3, dist3, rerank, entry
    int32_t* pool1_ids;  // nq x ef: C after stage (1), original ids
    float* pool1_dists;  // nq x ef: reduced-space FP32 distances
    int32_t* pool2_ids;  // nq x ef: C after re-rank + stage (2)
    float* pool2_dists;  // nq x ef: full-vector FP32 distances
};

// ------------------------------------------------------- number formats --

// BF16 -> FP64: a BF16 value is the upper 16 bits of an IEEE binary32.
double decode_bf16(uint16_t h) {
    uint32_t bits = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &bits, 4);
    return double(f);
}

// FP8 E4M3 "fn" -> FP64 from the format definition: 1 sign bit, 4 exponent
// bits (bias 7), 3 mantissa bits, subnormals when the exponent field is 0,
// and S.1111.111 the only NaN (no infinities).
double decode_e4m3(uint8_t c) {
    int sign = (c >> 7) & 1;
    int e = (c >> 3) & 0xF;
    int m = c & 7;
    double v;
    if (e == 0xF && m == 7) return NAN;
    if (e == 0) v = std::ldexp(double(m) / 8.0, 1 - 7);
    else v = std::ldexp(1.0 + double(m) / 8.0, e - 7);
    return sign ? -v : v;
}

// ------------------------------------------------------------ distances --

// Exact-then-round: the FP64 value of the distance, rounded once to FP32.
// Squared Euclidean for metric 0 (Sec. 5, Table 2 "squared euclidean");
// negated inner product for metric 1 so that smaller is closer.
float finish(double s, int metric) {
    float f = float(metric == 0 ? s : -s);
    if (f == 0.0f) f = 0.0f;  // -0.0 compares as +0.0
    return f;
}

double accumulate(const double* q, const double* x, int64_t d, int metric) {
    double s = 0.0;
    for (int64_t i = 0; i < d; ++i) {
        if (metric == 0) {
            double t = q[i] - x[i];
            s += t * t;
        } else {
            s += q[i] * x[i];
        }
    }
    return s;
}

struct Cand {
    float dist;
    int32_t id;      // original node id
    bool checked;
};

bool cand_less(const Cand& a, const Cand& b) {
    if (a.dist != b.dist) return a.dist < b.dist;
    return a.id < b.id;
}

struct Counters {
    int32_t exp = 0, dist = 0;
};

// One query's view of the index.
struct Searcher {
    const Index& ix;
    std::vector<int64_t> reduced_row;   // original id -> reduced row (-1 if unsampled)

    explicit Searcher(const Index& index) : ix(index), reduced_row(index.n, -1) {
        int64_t r = 0;
        for (int64_t v = 0; v < ix.n; ++v)
            if (ix.subgraph_mask[v]) reduced_row[v] = r++;
    }

    // Decoded reduced row of original node v (x_primary, Sec. 4.1 (1)).
    void reduced_vec(int32_t v, double* out) const {
        int64_t r = reduced_row[v];
        for (int64_t c = 0; c < ix.dp; ++c) {
            int64_t at = r * ix.dp + c;
            if (ix.reduced_dtype == 0) out[c] = double(((const float*)ix.reduced)[at]);
            else if (ix.reduced_dtype == 1) out[c] = decode_bf16(((const uint16_t*)ix.reduced)[at]);
            else out[c] = decode_e4m3(((const uint8_t*)ix.reduced)[at]) * double(ix.reduced_scales[r]);
        }
    }

    float reduced_dist(const double* qp, int32_t v, double* tmp) const {
        reduced_vec(v, tmp);
        return finish(accumulate(qp, tmp, ix.dp, ix.metric), ix.metric);
    }

    // Reduced-space distance from q' to coarse-cluster centroid c.
    float centroid_dist(const double* qp, int64_t c, double* tmp) const {
        for (int64_t i = 0; i < ix.dp; ++i) tmp[i] = double(ix.centroids[c * ix.dp + i]);
        return finish(accumulate(qp, tmp, ix.dp, ix.metric), ix.metric);
    }

    float full_dist(const double* q, int32_t v, double* tmp) const {
        const float* x = ix.full + int64_t(v) * ix.d;
        for (int64_t i = 0; i < ix.d; ++i) tmp[i] = double(x[i]);
        return finish(accumulate(q, tmp, ix.d, ix.metric), ix.metric);
    }
};

// Algorithm 1 (Sec. 2.2), "ANNS by Greedy Search": repeatedly take the first
// unchecked node u of the candidate list C, compute distances to u's
// unvisited neighbours (marking them visited), insert them into C, then
// shrink C to its ef best.  Stops when C has no unchecked node or after
// max_exp expansions (stage (2) runs a fixed number of them, Sec. 4.1 (2)).
// C is kept sorted by (distance, id).
template <class Neighbours, class Distance>
void greedy_search(std::vector<Cand>& C, std::vector<uint8_t>& visited, int64_t width,
                   Neighbours nbr, Distance dist, int ef, int64_t max_exp, Counters& cnt) {
    for (int64_t step = 0; step < max_exp; ++step) {
        size_t ui = C.size();
        for (size_t i = 0; i < C.size(); ++i)
            if (!C[i].checked) { ui = i; break; }
        if (ui == C.size()) break;           // no unchecked node left
        C[ui].checked = true;
        int32_t u = C[ui].id;
        cnt.exp += 1;
        const int32_t* row = nbr(u);
        for (int64_t j = 0; j < width; ++j) {
            int32_t v = row[j];
            if (v < 0 || visited[v]) continue;
            visited[v] = 1;
            float dv = dist(v);
            cnt.dist += 1;
            C.push_back(Cand{dv, v, false});
        }
        std::sort(C.begin(), C.end(), cand_less);
        if (C.size() > size_t(ef)) C.resize(size_t(ef));
    }
}

// Projection onto the leading dp right singular vectors, q' = q V[:, :dp]
// (Sec. 4.1 (1): x_primary = U_{1..d'} Sigma_{1..d'} = x V_{1..d'}), in FP64.
void project(const Index& ix, const float* q, double* qp) {
    for (int64_t c = 0; c < ix.dp; ++c) {
        double s = 0.0;
        for (int64_t j = 0; j < ix.d; ++j) s += double(q[j]) * ix.basis[j * ix.dp + c];
        qp[c] = s;
    }
}

// The staged search of Sec. 4.1 for one query.
void search_one(const Searcher& S, const Params& P, const float* query, int64_t qi, const Outputs& out) {
    const Index& ix = S.ix;
    std::vector<double> q(ix.d), qp(ix.dp), tmp(std::max(ix.d, ix.dp));
    for (int64_t i = 0; i < ix.d; ++i) q[i] = double(query[i]);

    // Stage (1) input: the projected query, stored at the paper's FP32.
    project(ix, query, qp.data());
    for (int64_t c = 0; c < ix.dp; ++c) qp[c] = double(float(qp[c]));

    // Fast entry selection, dense form (Sec. 5 / Table 2 "FES (1 block)"):
    // the entry vectors closest to q' by (distance, id) seed stage (1).  The
    // paper seeds with the single closest one (fes_seeds = 1); more seeds are
    // the top-T variant.  Without FES the seeds are the first entries of the
    // set.  At most ef seeds.
    //
    // Clustered FES (Sec. 5, "clustering-based selection"): the query goes to
    // the coarse cluster whose centroid is closest by (distance, cluster
    // index), and only that cluster's entries are scored.
    std::vector<Cand> seeds;
    if (P.use_fes == 2) {
        int64_t best_c = 0;
        float best_d = 0.0f;
        for (int64_t c = 0; c < ix.n_clusters; ++c) {
            const float dc = S.centroid_dist(qp.data(), c, tmp.data());
            if (c == 0 || dc < best_d) { best_d = dc; best_c = c; }
        }
        for (int64_t e = 0; e < ix.n_entry; ++e)
            if (ix.entry_cluster[e] == best_c)
                seeds.push_back(Cand{S.reduced_dist(qp.data(), ix.entry_ids[e], tmp.data()), ix.entry_ids[e], false});
    } else {
        const int64_t n_scored =
            P.use_fes ? ix.n_entry : std::min<int64_t>(std::min<int64_t>(P.fes_seeds, P.ef), ix.n_entry);
        for (int64_t e = 0; e < n_scored; ++e)
            seeds.push_back(Cand{S.reduced_dist(qp.data(), ix.entry_ids[e], tmp.data()), ix.entry_ids[e], false});
    }
    std::sort(seeds.begin(), seeds.end(), cand_less);
    const int64_t ns = std::min<int64_t>(std::min<int64_t>(P.fes_seeds, P.ef), int64_t(seeds.size()));
    seeds.resize(size_t(ns));
    const Cand entry = seeds[0];

    Counters c1, c2, c3;
    std::vector<uint8_t> visited(ix.n, 0);

    // The experiment of Sec. 4.2: the final stage alone (Algorithm 1 on the
    // full graph), its candidate list seeded with given nodes (known true
    // neighbours plus random ones), all unchecked and visited.
    if (P.seed_ids) {
        std::vector<Cand> C;
        int32_t scored = 0;
        for (int j = 0; j < P.seed_count; ++j) {
            const int32_t v = P.seed_ids[qi * P.seed_count + j];
            if (v < 0 || visited[v]) continue;
            visited[v] = 1;
            C.push_back(Cand{S.full_dist(q.data(), v, tmp.data()), v, false});
            scored += 1;
        }
        std::sort(C.begin(), C.end(), cand_less);
        if (C.size() > size_t(P.ef)) C.resize(size_t(P.ef));
        greedy_search(C, visited, ix.R, [&](int32_t u) { return ix.graph + int64_t(u) * ix.R; },
                      [&](int32_t v) { return S.full_dist(q.data(), v, tmp.data()); }, P.ef, INT64_MAX, c3);
        for (int j = 0; j < P.k; ++j) {
            const bool ok = size_t(j) < C.size();
            if (out.ids) out.ids[qi * P.k + j] = ok ? C[j].id : -1;
            if (out.dists) out.dists[qi * P.k + j] = ok ? C[j].dist : INFINITY;
        }
        if (out.counters) {
            int32_t* k = out.counters + qi * 8;
            k[0] = k[1] = k[2] = k[3] = 0;
            k[4] = c3.exp; k[5] = c3.dist; k[6] = scored; k[7] = -1;
        }
        return;
    }

    // Stage (1): Algorithm 1 over the subgraph with reduced distances, from
    // the seeds (all unchecked, all visited).
    std::vector<Cand> C = seeds;
    for (const Cand& c : C) visited[c.id] = 1;
    if (P.stage1) {
        greedy_search(C, visited, ix.R_sub,
                      [&](int32_t u) { return ix.subgraph + int64_t(u) * ix.R_sub; },
                      [&](int32_t v) { return S.reduced_dist(qp.data(), v, tmp.data()); },
                      P.ef, INT64_MAX, c1);
    }
    if (out.pool1_ids) {
        for (int j = 0; j < P.ef; ++j) {
            bool ok = size_t(j) < C.size();
            out.pool1_ids[qi * P.ef + j] = ok ? C[j].id : -1;
            out.pool1_dists[qi * P.ef + j] = ok ? C[j].dist : INFINITY;
        }
    }

    // Stage (2), part 1: full-vector distances for every candidate of stage
    // (1), a fresh visited table holding exactly those candidates, C
    // re-sorted and all candidates unchecked (Sec. 4.1 (2)).
    int32_t n_rerank = 0;
    std::fill(visited.begin(), visited.end(), 0);
    for (Cand& c : C) {
        c.dist = S.full_dist(q.data(), c.id, tmp.data());
        c.checked = false;
        visited[c.id] = 1;
        n_rerank += 1;
    }
    std::sort(C.begin(), C.end(), cand_less);

    // Stage (2), part 2: a fixed, small number of expansions on the subgraph
    // with full-vector distances (the paper uses 2).
    greedy_search(C, visited, ix.R_sub,
                  [&](int32_t u) { return ix.subgraph + int64_t(u) * ix.R_sub; },
                  [&](int32_t v) { return S.full_dist(q.data(), v, tmp.data()); },
                  P.ef, P.stage2_expansions, c2);
    if (out.pool2_ids) {
        for (int j = 0; j < P.ef; ++j) {
            bool ok = size_t(j) < C.size();
            out.pool2_ids[qi * P.ef + j] = ok ? C[j].id : -1;
            out.pool2_dists[qi * P.ef + j] = ok ? C[j].dist : INFINITY;
        }
    }

    // Stage (3): Algorithm 1 over the full graph with full vectors, seeded by
    // stage (2)'s candidates and reusing its visited table.  No candidate has
    // been expanded on the full graph yet, so all start unchecked.
    if (P.stage3) {
        for (Cand& c : C) c.checked = false;
        greedy_search(C, visited, ix.R,
                      [&](int32_t u) { return ix.graph + int64_t(u) * ix.R; },
                      [&](int32_t v) { return S.full_dist(q.data(), v, tmp.data()); },
                      P.ef, INT64_MAX, c3);
    }

    // Output: the first k of C by (distance, id).
    if (out.ids) {
        for (int j = 0; j < P.k; ++j) {
            bool ok = size_t(j) < C.size();
            out.ids[qi * P.k + j] = ok ? C[j].id : -1;
            out.dists[qi * P.k + j] = ok ? C[j].dist : INFINITY;
        }
    }
    if (out.counters) {
        int32_t* k = out.counters + qi * 8;
        k[0] = c1.exp; k[1] = c1.dist; k[2] = c2.exp; k[3] = c2.dist;
        k[4] = c3.exp; k[5] = c3.dist; k[6] = n_rerank; k[7] = entry.id;
    }
}

template <class F>
void parallel_for(int64_t n, int nthreads, F f) {
    if (nthreads <= 1 || n <= 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&, t] {
            for (int64_t i = t; i < n; i += nthreads) f(i);
        });
    for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

// Staged search of Sec. 4.1 over nq queries (nq x d FP32, row-major).
// Returns 0 on success, -1 on invalid arguments.
int oracle_search(const Index* ix, const Params* P, const float* queries, int64_t nq, const Outputs* out) {
    if (!ix || !P || P->k < 1 || P->ef < P->k || ix->n_entry < 1 || P->fes_seeds < 1) return -1;
    if (P->use_fes == 2) {   // every cluster must hold an entry
        if (ix->n_clusters < 1 || !ix->entry_cluster || !ix->centroids) return -1;
        std::vector<int64_t> size(size_t(ix->n_clusters), 0);
        for (int64_t e = 0; e < ix->n_entry; ++e) {
            if (ix->entry_cluster[e] < 0 || ix->entry_cluster[e] >= ix->n_clusters) return -1;
            size[size_t(ix->entry_cluster[e])] += 1;
        }
        for (int64_t c : size)
            if (c == 0) return -1;
    }
    Searcher S(*ix);
    parallel_for(nq, P->nthreads, [&](int64_t qi) { search_one(S, *P, queries + qi * ix->d, qi, *out); });
    return 0;
}

// q' = round_FP32(q V[:, :dp]) per component, plus the unrounded FP64 value.
int oracle_project(const Index* ix, const float* queries, int64_t nq, double* out_f64, float* out_f32) {
    std::vector<double> qp(ix->dp);
    for (int64_t qi = 0; qi < nq; ++qi) {
        project(*ix, queries + qi * ix->d, qp.data());
        for (int64_t c = 0; c < ix->dp; ++c) {
            if (out_f64) out_f64[qi * ix->dp + c] = qp[c];
            if (out_f32) out_f32[qi * ix->dp + c] = float(qp[c]);
        }
    }
    return 0;
}

// Dense FES alone: for each projected query (nq x dp FP32), the entry with
// the smallest (FP32 distance, id) and that distance.
int oracle_fes(const Index* ix, const float* qproj, int64_t nq, int32_t* out_entry, float* out_dist) {
    Searcher S(*ix);
    std::vector<double> qp(ix->dp), tmp(ix->dp);
    for (int64_t qi = 0; qi < nq; ++qi) {
        for (int64_t c = 0; c < ix->dp; ++c) qp[c] = double(qproj[qi * ix->dp + c]);
        Cand best{INFINITY, -1, false};
        for (int64_t e = 0; e < ix->n_entry; ++e) {
            Cand c{S.reduced_dist(qp.data(), ix->entry_ids[e], tmp.data()), ix->entry_ids[e], false};
            if (best.id < 0 || cand_less(c, best)) best = c;
        }
        out_entry[qi] = best.id;
        out_dist[qi] = best.dist;
    }
    return 0;
}

// Exact FP64 brute-force top-k over the full vectors (recall ground truth,
// Sec. 6.1 "Metrics"): smallest (FP64 distance, id), distances in FP64.
int oracle_bruteforce(const float* base, int64_t n, int64_t d, int metric, const float* queries, int64_t nq,
                      int k, int nthreads, int32_t* out_ids, double* out_dists) {
    parallel_for(nq, nthreads, [&](int64_t qi) {
        std::vector<std::pair<double, int32_t>> all(n);
        const float* q = queries + qi * d;
        for (int64_t v = 0; v < n; ++v) {
            const float* x = base + v * d;
            double s = 0.0;
            for (int64_t i = 0; i < d; ++i) {
                if (metric == 0) {
                    double t = double(q[i]) - double(x[i]);
                    s += t * t;
                } else {
                    s += double(q[i]) * double(x[i]);
                }
            }
            all[v] = {metric == 0 ? s : -s, int32_t(v)};
        }
        int kk = int(std::min<int64_t>(k, n));
        std::partial_sort(all.begin(), all.begin() + kk, all.end());
        for (int j = 0; j < k; ++j) {
            out_ids[qi * k + j] = j < kk ? all[j].second : -1;
            out_dists[qi * k + j] = j < kk ? all[j].first : INFINITY;
        }
    });
    return 0;
}

// Exposed decoders so the tests can pin them against the format tables.
double oracle_decode_e4m3(uint8_t c) { return decode_e4m3(c); }
double oracle_decode_bf16(uint16_t h) { return decode_bf16(h); }

int oracle_abi_version(void) { return 1; }

}  // extern "C"
