// serve.cu -- continuous-batching search server (pilot_serve_* in pilot.h).
//
// A background thread drives K CUDA streams ("lanes"), each with its own
// sequence of steps.  A step admits queued requests into free slots (slot
// count set by the HBM budget, ef bounded by the shared-memory budget of the
// step kernel), projects and scores the new requests' FES candidates, and
// replays a CUDA graph holding the step kernel: every request of the step
// advances by at most `expansions_per_step` expansions of the staged search,
// keeping its candidate list, visited table and phase in device memory.
// Finished requests write their top-k to host-mapped memory; the thread
// completes their tickets and records submit-to-completion latency.
//
// A request stays on the lane that admitted it until it finishes: one that
// outlives its step is listed again in the lane's next step, so steps that
// run at the same time on different lanes hold disjoint slots.  Requests that
// arrive while steps run are admitted by the next idle lane, so their work
// overlaps on the device with the steps in flight and no step waits for
// another's tail.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pilot.h"
#include "kernels.h"

namespace pilot {
IndexView index_view(pilot_index* ix);
int set_error(int status, const char* msg);
}  // namespace pilot

using namespace pilot;

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
    return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

pilot_status err(pilot_status s, const char* fmt, long long a = 0, long long b = 0) {
    char buf[400];
    snprintf(buf, sizeof buf, fmt, a, b);
    return pilot_status(set_error(int(s), buf));
}

pilot_status cuda_err(cudaError_t e, const char* what) {
    cudaGetLastError();
    char buf[300];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return pilot_status(set_error(int(e == cudaErrorMemoryAllocation ? PILOT_ENOMEM : PILOT_ECUDA), buf));
}

struct Request {
    uint64_t ticket;
    int k, ef;
    double t_submit;
    std::vector<float> q;
};

struct Result {
    pilot_status status;
    std::vector<int32_t> ids;
    std::vector<float> dists;
    int32_t counters[8];
};

}  // namespace

struct pilot_server {
    pilot_index* index = nullptr;
    IndexView view{};
    DevIndex X{};
    pilot_serve_config cfg{};
    SearchConfig scfg{};
    int slots = 0;

    // One stream with its own step sequence: its step graph, host-mapped
    // entry list, and buffers for the requests it admits.
    struct Lane {
        cudaStream_t stream = nullptr;
        cudaGraphExec_t graph = nullptr;
        cudaEvent_t done = nullptr;
        bool in_flight = false;
        double t_launch = 0.0;
        ServeEntry* entries = nullptr;    // host-mapped, one per slot at most
        int32_t* n_active = nullptr;      // host-mapped
        int32_t* next = nullptr;          // device counter, zeroed by the graph
        float* staging_q = nullptr;       // pinned, new requests' vectors
        float *new_q = nullptr, *new_q_pad = nullptr, *new_qp = nullptr;
        int32_t *new_pos = nullptr, *new_bad = nullptr, *new_status = nullptr;
        uint16_t* new_qpb = nullptr;
        double* new_lb = nullptr;
        std::vector<int> owned;           // slots whose requests run on this lane
    };
    std::vector<Lane> lanes;

    // device state, one entry per slot
    std::vector<void*> dev_allocs;
    std::vector<void*> host_allocs;
    SlotState* state = nullptr;
    uint64_t* pool = nullptr;
    float *q_pad = nullptr, *qp = nullptr;
    uint16_t* vis = nullptr;          // per slot, vis_stride words (sized by max_ef and the degree)
    int64_t vis_stride = 0;
    int32_t* vis_overflow = nullptr;  // device counter
    int32_t *res_ids = nullptr, *res_done = nullptr, *res_counters = nullptr;   // host-mapped
    float* res_dists = nullptr;

    // host state
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Result> results;
    std::vector<Request> slot_req;      // request occupying each slot
    std::vector<int> free_slots;
    uint64_t next_ticket = 1;
    bool stop = false;
    pilot_status broken = PILOT_OK;
    // stats
    uint64_t submitted = 0, admitted = 0, rejected = 0, completed = 0, steps = 0;
    double t_first_submit = -1, t_last_done = -1;
    std::vector<double> latencies;

    template <class T>
    pilot_status dalloc(T** p, size_t count) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, std::max<size_t>(count * sizeof(T), 16));
        if (e != cudaSuccess) return cuda_err(e, "cudaMalloc (server)");
        dev_allocs.push_back(v);
        *p = static_cast<T*>(v);
        return PILOT_OK;
    }
    template <class T>
    pilot_status halloc(T** p, size_t count) {
        void* v = nullptr;
        cudaError_t e = cudaHostAlloc(&v, std::max<size_t>(count * sizeof(T), 16), cudaHostAllocMapped);
        if (e != cudaSuccess) return cuda_err(e, "cudaHostAlloc (server)");
        host_allocs.push_back(v);
        std::memset(v, 0, std::max<size_t>(count * sizeof(T), 16));
        *p = static_cast<T*>(v);
        return PILOT_OK;
    }

    ~pilot_server() {
        for (Lane& L : lanes)
            if (L.stream) cudaStreamSynchronize(L.stream);
        for (Lane& L : lanes) {
            if (L.graph) cudaGraphExecDestroy(L.graph);
            if (L.done) cudaEventDestroy(L.done);
            if (L.stream) cudaStreamDestroy(L.stream);
        }
        for (void* p : dev_allocs) cudaFree(p);
        for (void* p : host_allocs) cudaFreeHost(p);
    }

    size_t in_flight_requests() const {
        size_t n = 0;
        for (const Lane& L : lanes) n += L.owned.size();
        return n;
    }
    void loop();
    pilot_status enqueue(int k, bool* launched);
    pilot_status complete(int k);
    void fail_all(pilot_status s);
};

// Fail every request still owned by a lane or waiting (after an error).
void pilot_server::fail_all(pilot_status s) {
    for (Lane& L : lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    std::lock_guard<std::mutex> lk(mu);
    broken = s;
    for (Lane& L : lanes) {
        L.in_flight = false;
        for (int slot : L.owned) results[slot_req[size_t(slot)].ticket] = Result{s, {}, {}, {}};
        L.owned.clear();
    }
    for (Request& r : queue) results[r.ticket] = Result{s, {}, {}, {}};
    queue.clear();
    cv_done.notify_all();
}

void pilot_server::loop() {
    cudaSetDevice(view.device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            bool busy = false;
            for (const Lane& L : lanes) busy = busy || L.in_flight;
            if (!busy && queue.empty() && in_flight_requests() == 0)
                cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop || !queue.empty(); });
            if (stop) return;
            if (broken != PILOT_OK) {   // fail everything still pending
                for (Request& r : queue) results[r.ticket] = Result{broken, {}, {}, {}};
                queue.clear();
                cv_done.notify_all();
                continue;
            }
        }
        bool progress = false;
        pilot_status s = PILOT_OK;
        // finished steps first: they free slots for the launches below
        for (int k = 0; k < int(lanes.size()) && s == PILOT_OK; ++k) {
            Lane& L = lanes[size_t(k)];
            if (!L.in_flight) continue;
            const cudaError_t e = cudaEventQuery(L.done);
            if (e == cudaSuccess) {
                s = complete(k);
                progress = true;
            } else if (e != cudaErrorNotReady) {
                s = cuda_err(e, "serving step");
            } else if (now_ms() - L.t_launch > double(cfg.step_timeout_ms)) {
                s = err(PILOT_ETIMEOUT, "a serving step ran longer than %lld ms", (long long)cfg.step_timeout_ms);
            }
        }
        for (int k = 0; k < int(lanes.size()) && s == PILOT_OK; ++k) {
            if (lanes[size_t(k)].in_flight) continue;
            bool launched = false;
            s = enqueue(k, &launched);
            progress = progress || launched;
        }
        if (s != PILOT_OK) {
            fail_all(s);
            continue;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Prepare and launch a step on lane k: the lane's unfinished requests plus
// queued requests admitted into free slots; upload, project and score the new
// ones, and replay the lane's step graph.  Nothing is launched when the lane
// has nothing to run.
pilot_status pilot_server::enqueue(int k, bool* launched) {
    *launched = false;
    Lane& L = lanes[size_t(k)];
    int n_new = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        int n = 0;
        const int cap_new = std::min<int>(int(free_slots.size()), cfg.max_new_per_step);
        ServeEntry* E = L.entries;
        while (!queue.empty() && n_new < cap_new) {
            Request r = std::move(queue.front());
            queue.pop_front();
            const int slot = free_slots.back();
            free_slots.pop_back();
            std::memcpy(L.staging_q + size_t(n_new) * size_t(X.d), r.q.data(), size_t(X.d) * 4);
            reinterpret_cast<volatile int32_t*>(res_done)[slot] = 0;
            E[n++] = ServeEntry{slot, n_new, r.k, r.ef};
            r.q.clear();
            slot_req[size_t(slot)] = std::move(r);
            ++n_new;
            ++admitted;
        }
        for (int slot : L.owned) E[n++] = ServeEntry{slot, -1, slot_req[size_t(slot)].k, slot_req[size_t(slot)].ef};
        for (int i = 0; i < n_new; ++i) L.owned.push_back(E[i].slot);
        *reinterpret_cast<volatile int32_t*>(L.n_active) = n;
        if (n == 0) return PILOT_OK;
    }
    cudaError_t e;
    if (n_new > 0) {
        if ((e = cudaMemcpyAsync(L.new_q, L.staging_q, size_t(n_new) * size_t(X.d) * 4, cudaMemcpyHostToDevice,
                                 L.stream)) != cudaSuccess)
            return cuda_err(e, "copy new requests");
        if ((e = cudaMemsetAsync(L.new_status, 0, 8 * 4, L.stream)) != cudaSuccess) return cuda_err(e, "clear status");
        SearchIO io{};
        io.nq = n_new;
        io.queries = L.new_q;
        io.q_pad = L.new_q_pad;
        io.qp = L.new_qp;
        io.fes_pos = L.new_pos;
        io.qp_bf16 = L.new_qpb;
        io.fes_lb = L.new_lb;
        io.bad_query = L.new_bad;
        io.status = L.new_status;
        if ((e = launch_project(X, io, L.stream)) != cudaSuccess) return cuda_err(e, "projection kernel");
        if (scfg.use_fes && (e = launch_fes_mma(X, io, L.stream)) != cudaSuccess)
            return cuda_err(e, "FES tensor-core kernel");
    }
    if ((e = cudaGraphLaunch(L.graph, L.stream)) != cudaSuccess) return cuda_err(e, "step graph");
    if ((e = cudaEventRecord(L.done, L.stream)) != cudaSuccess) return cuda_err(e, "record step");
    L.in_flight = true;
    L.t_launch = now_ms();
    *launched = true;
    return PILOT_OK;
}

// Complete every request of lane k's finished step whose done flag is raised;
// the others stay with the lane for its next step.
pilot_status pilot_server::complete(int k) {
    Lane& L = lanes[size_t(k)];
    L.in_flight = false;
    const double t = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    ++steps;
    std::vector<int> still;
    still.reserve(L.owned.size());
    for (int slot : L.owned) {
        const int done = reinterpret_cast<volatile int32_t*>(res_done)[slot];
        if (!done) {
            still.push_back(slot);
            continue;
        }
        Request& r = slot_req[size_t(slot)];
        Result res;
        res.status = done == 1 ? PILOT_OK : PILOT_ETIMEOUT;
        res.ids.assign(res_ids + size_t(slot) * size_t(cfg.max_k), res_ids + size_t(slot) * size_t(cfg.max_k) + r.k);
        res.dists.assign(res_dists + size_t(slot) * size_t(cfg.max_k),
                         res_dists + size_t(slot) * size_t(cfg.max_k) + r.k);
        for (int i = 0; i < 8; ++i) res.counters[i] = reinterpret_cast<volatile int32_t*>(res_counters)[slot * 8 + i];
        results[r.ticket] = std::move(res);
        latencies.push_back(t - r.t_submit);
        t_last_done = t;
        ++completed;
        free_slots.push_back(slot);
    }
    L.owned.swap(still);
    cv_done.notify_all();
    return PILOT_OK;
}

extern "C" {

void pilot_serve_config_default(pilot_serve_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->max_slots = 16384;
    c->max_ef = 512;
    c->max_k = 100;
    c->expansions_per_step = 4096;
    c->max_new_per_step = 8192;
    c->queue_capacity = 1 << 20;
    c->step_timeout_ms = 10000;
    c->streams = 4;
}

pilot_status pilot_serve_create(pilot_index* index, const pilot_serve_config* config, pilot_server** out) {
    if (!index || !out) return err(PILOT_EINVAL, "index and out must not be NULL");
    *out = nullptr;
    pilot_serve_config c;
    pilot_serve_config_default(&c);
    if (config) c = *config;
    if (c.max_ef < 1 || c.max_ef > PILOT_MAX_EF) return err(PILOT_EINVAL, "max_ef must be in [1, %lld]", PILOT_MAX_EF);
    if (c.max_k < 1 || c.max_k > c.max_ef) return err(PILOT_EINVAL, "max_k must be in [1, max_ef]");
    if (c.expansions_per_step < 1) return err(PILOT_EINVAL, "expansions_per_step must be >= 1");
    if (c.max_new_per_step < 1 || c.queue_capacity < 1 || c.step_timeout_ms < 1 || c.max_slots < 1)
        return err(PILOT_EINVAL, "max_slots, max_new_per_step, queue_capacity and step_timeout_ms must be >= 1");
    if (c.streams == 0) c.streams = 4;
    if (c.streams < 1 || c.streams > 16) return err(PILOT_EINVAL, "streams = %lld must be in [1, 16]", c.streams);
    auto* S = new pilot_server();
    std::unique_ptr<pilot_server> guard(S);
    S->index = index;
    S->view = index_view(index);
    S->X = *S->view.dev;
    S->cfg = c;
    cudaError_t e = cudaSetDevice(S->view.device);
    if (e != cudaSuccess) return cuda_err(e, "cudaSetDevice");
    const DevIndex& X = S->X;

    // shared-memory budget: the step kernel's per-block slice for max_ef
    S->scfg = default_search_config(X, c.max_k, c.max_ef);
    {   // the autotuned staging rows of max_ef's class, if the index has them;
        // the step kernel keeps two warps per block whatever the tuner chose
        // for whole batches: the lanes' step kernels run side by side, and
        // small blocks share the SMs' shared memory between them more finely
        // (served capacity on the 1M x 96 index fell from 418k to 306k
        // requests/s with the 8-warp blocks a batch tuning picked)
        std::lock_guard<std::mutex> lock(*static_cast<std::mutex*>(S->view.mutex));
        const TunedShape t = S->view.tuned[ef_class(int(c.max_ef))];
        if (t.stage_rows > 0) set_stage_rows(X, S->scfg, t.stage_rows);
    }
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, S->view.device);
    if (serve_smem_per_block(X, S->scfg) > size_t(smem_max))
        return err(PILOT_EINVAL, "max_ef = %lld needs more shared memory per block than the device has",
                   (long long)c.max_ef);

    // HBM budget: per slot its list, query rows, state and visited table
    // (sized by max_ef and the degree, independent of n)
    const int pool_stride = [&] { int p = 32; while (p < c.max_ef) p <<= 1; return p; }();
    S->vis_stride = vis_entries_for(int(c.max_ef), std::max(X.R, X.R_sub), X.id_bits);
    const size_t per_slot = size_t(pool_stride) * 8 + size_t(X.d_pad + X.qp_pad) * 4 + sizeof(SlotState) +
                            size_t(S->vis_stride) * sizeof(uint16_t);
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda_err(e, "cudaMemGetInfo");
    const size_t budget = c.hbm_budget_bytes > 0 ? size_t(c.hbm_budget_bytes) : free_b / 4;
    const int64_t fit = int64_t(budget / per_slot);
    S->slots = int(std::min<int64_t>(c.max_slots, fit));
    if (S->slots < 1) return err(PILOT_ENOMEM, "the HBM budget holds no slot (%lld bytes per slot)", (long long)per_slot);
    {   // whole waves: a multiple of the step kernel's resident warps, so no step ends on a partial wave
        int all_blocks = 0;
        size_t smem_probe = 0;
        if ((e = prepare_serve_step(X, S->scfg, S->view.num_sms, 1 << 30, &all_blocks, &smem_probe)) != cudaSuccess)
            return cuda_err(e, "size the step kernel");
        const int resident = all_blocks * S->scfg.warps_per_block;
        if (resident > 0 && S->slots >= resident) S->slots -= S->slots % resident;
    }
    const int NS = S->slots, NN = std::min<int>(c.max_new_per_step, S->slots);
    S->cfg.max_new_per_step = NN;

    pilot_status ps;
    if ((ps = S->dalloc(&S->state, size_t(NS))) != PILOT_OK) return ps;
    if ((ps = S->dalloc(&S->pool, size_t(NS) * pool_stride)) != PILOT_OK) return ps;
    if ((ps = S->dalloc(&S->q_pad, size_t(NS) * X.d_pad)) != PILOT_OK) return ps;
    if ((ps = S->dalloc(&S->qp, size_t(NS) * X.qp_pad)) != PILOT_OK) return ps;
    if ((ps = S->dalloc(&S->vis, size_t(NS) * size_t(S->vis_stride))) != PILOT_OK) return ps;
    if ((ps = S->dalloc(&S->vis_overflow, 1)) != PILOT_OK) return ps;
    if ((e = cudaMemset(S->state, 0, size_t(NS) * sizeof(SlotState))) != cudaSuccess) return cuda_err(e, "clear");
    if ((e = cudaMemset(S->vis, 0, size_t(NS) * size_t(S->vis_stride) * sizeof(uint16_t))) != cudaSuccess)
        return cuda_err(e, "clear");
    if ((e = cudaMemset(S->vis_overflow, 0, 4)) != cudaSuccess) return cuda_err(e, "clear");
    if ((ps = S->halloc(&S->res_ids, size_t(NS) * c.max_k)) != PILOT_OK) return ps;
    if ((ps = S->halloc(&S->res_dists, size_t(NS) * c.max_k)) != PILOT_OK) return ps;
    if ((ps = S->halloc(&S->res_done, size_t(NS))) != PILOT_OK) return ps;
    if ((ps = S->halloc(&S->res_counters, size_t(NS) * 8)) != PILOT_OK) return ps;

    // the lanes: each its own stream, buffers for the requests it admits and a
    // step graph (reset the lane's slot counter, run the step kernel)
    ServeIO sio{};
    sio.state = S->state;
    sio.pool = S->pool;
    sio.pool_stride = pool_stride;
    sio.q_pad = S->q_pad;
    sio.qp = S->qp;
    sio.res_ids = S->res_ids;
    sio.res_dists = S->res_dists;
    sio.res_done = S->res_done;
    sio.res_counters = S->res_counters;
    sio.k_max = c.max_k;
    sio.budget = c.expansions_per_step;
    DevIndex XS = X;
    XS.vis = S->vis;   // the server's own visited tables, one per slot
    XS.vis_stride = S->vis_stride;
    XS.vis_slots = NS;
    XS.vis_epoch = nullptr;   // slots keep their epoch counters in SlotState
    set_visited_size(XS, S->scfg, S->vis_stride);
    sio.vis = S->vis;
    sio.vis_overflow = S->vis_overflow;
    int blocks = 0;
    size_t smem = 0;
    if ((e = prepare_serve_step(XS, S->scfg, S->view.num_sms, NS, &blocks, &smem)) != cudaSuccess)
        return cuda_err(e, "size the step kernel");
    S->lanes.resize(size_t(c.streams));
    for (pilot_server::Lane& L : S->lanes) {
        if ((ps = S->halloc(&L.entries, size_t(NS))) != PILOT_OK) return ps;
        if ((ps = S->halloc(&L.n_active, 1)) != PILOT_OK) return ps;
        if ((ps = S->halloc(&L.staging_q, size_t(NN) * X.d)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.next, 1)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_q, size_t(NN) * X.d)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_q_pad, size_t(NN) * X.d_pad)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_qp, size_t(NN) * X.qp_pad)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_pos, size_t(NN) * S->scfg.fes_T)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_qpb, size_t((NN + 127) / 128 * 128) * X.qp_pad)) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_lb, size_t(NN))) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_bad, size_t(NN))) != PILOT_OK) return ps;
        if ((ps = S->dalloc(&L.new_status, 8)) != PILOT_OK) return ps;
        if ((e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_err(e, "cudaEventCreate");
        if ((e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_err(e, "cudaStreamCreate");
        sio.entries = L.entries;
        sio.n_active = L.n_active;
        sio.next = L.next;
        sio.new_q_pad = L.new_q_pad;
        sio.new_qp = L.new_qp;
        sio.new_fes_pos = L.new_pos;
        sio.new_fes_lb = L.new_lb;
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_err(e, "begin capture");
        cudaError_t e1 = cudaMemsetAsync(L.next, 0, 4, L.stream);
        cudaError_t e2 = launch_serve_step(XS, S->scfg, sio, L.stream, blocks, smem);
        cudaError_t e3 = cudaStreamEndCapture(L.stream, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_err(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "capture step graph");
        }
        e = cudaGraphInstantiate(&L.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e, "instantiate step graph");
    }
    S->X = XS;

    S->slot_req.resize(size_t(NS));
    for (int i = NS - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->worker = std::thread([S] { S->loop(); });
    *out = guard.release();
    return PILOT_OK;
}

pilot_status pilot_serve_submit(pilot_server* s, const float* q, int k, int ef, uint64_t* ticket) {
    if (!s || !q || !ticket) return err(PILOT_EINVAL, "server, query and ticket must not be NULL");
    if (k < 1 || k > s->cfg.max_k) return err(PILOT_EINVAL, "k = %lld outside [1, max_k = %lld]", k, s->cfg.max_k);
    if (ef < k || ef > s->cfg.max_ef)
        return err(PILOT_EINVAL, "ef = %lld outside [k, max_ef = %lld]", ef, s->cfg.max_ef);
    for (int64_t i = 0; i < s->X.d; ++i)
        if (!std::isfinite(q[i])) return err(PILOT_EINVAL, "the query holds NaN or infinity");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken != PILOT_OK) return err(s->broken, "the server stopped after an error");
    if (int64_t(s->queue.size()) >= s->cfg.queue_capacity) {
        ++s->rejected;
        return err(PILOT_EBUSY, "the request queue is full (%lld waiting)", (long long)s->queue.size());
    }
    Request r;
    r.ticket = s->next_ticket++;
    r.k = k;
    r.ef = ef;
    r.t_submit = now_ms();
    r.q.assign(q, q + s->X.d);
    if (s->t_first_submit < 0) s->t_first_submit = r.t_submit;
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    ++s->submitted;
    s->cv_work.notify_one();
    return PILOT_OK;
}

pilot_status pilot_serve_submit_batch(pilot_server* s, const float* queries, int64_t n, const int32_t* k,
                                      const int32_t* ef, uint64_t* tickets) {
    if (!s || n < 0 || (n > 0 && (!queries || !k || !ef || !tickets)))
        return err(PILOT_EINVAL, "server, queries, k, ef and tickets must not be NULL");
    for (int64_t i = 0; i < n; ++i) {   // validate everything before queueing anything
        if (k[i] < 1 || k[i] > s->cfg.max_k)
            return err(PILOT_EINVAL, "request %lld: k outside [1, max_k = %lld]", (long long)i, s->cfg.max_k);
        if (ef[i] < k[i] || ef[i] > s->cfg.max_ef)
            return err(PILOT_EINVAL, "request %lld: ef outside [k, max_ef = %lld]", (long long)i, s->cfg.max_ef);
        const float* q = queries + i * s->X.d;
        for (int64_t j = 0; j < s->X.d; ++j)
            if (!std::isfinite(q[j])) return err(PILOT_EINVAL, "request %lld holds NaN or infinity", (long long)i);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken != PILOT_OK) return err(s->broken, "the server stopped after an error");
    if (int64_t(s->queue.size()) + n > s->cfg.queue_capacity) {
        s->rejected += uint64_t(n);
        return err(PILOT_EBUSY, "the request queue cannot take %lld more (%lld waiting)", (long long)n,
                   (long long)s->queue.size());
    }
    const double t = now_ms();
    if (s->t_first_submit < 0 && n > 0) s->t_first_submit = t;
    for (int64_t i = 0; i < n; ++i) {
        Request r;
        r.ticket = s->next_ticket++;
        r.k = k[i];
        r.ef = ef[i];
        r.t_submit = t;
        r.q.assign(queries + i * s->X.d, queries + (i + 1) * s->X.d);
        tickets[i] = r.ticket;
        s->queue.push_back(std::move(r));
    }
    s->submitted += uint64_t(n);
    s->cv_work.notify_one();
    return PILOT_OK;
}

pilot_status pilot_serve_wait(pilot_server* s, uint64_t ticket, int timeout_ms, int32_t* ids, float* dists) {
    return pilot_serve_wait_ex(s, ticket, timeout_ms, ids, dists, nullptr);
}

pilot_status pilot_serve_wait_ex(pilot_server* s, uint64_t ticket, int timeout_ms, int32_t* ids, float* dists,
                                 int32_t* counters) {
    if (!s) return err(PILOT_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        auto it = s->results.find(ticket);
        if (it != s->results.end()) {
            Result r = std::move(it->second);
            s->results.erase(it);
            lk.unlock();
            if (r.status != PILOT_OK) return err(r.status, "the request failed on the GPU");
            if (ids) std::memcpy(ids, r.ids.data(), r.ids.size() * 4);
            if (dists) std::memcpy(dists, r.dists.data(), r.dists.size() * 4);
            if (counters) std::memcpy(counters, r.counters, sizeof r.counters);
            return PILOT_OK;
        }
        if (ticket == 0 || ticket >= s->next_ticket) return err(PILOT_EINVAL, "unknown ticket %lld", (long long)ticket);
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !s->results.count(ticket))
            return err(PILOT_ETIMEOUT, "ticket %lld not done within %lld ms", (long long)ticket, timeout_ms);
    }
}

pilot_status pilot_serve_stats(pilot_server* s, pilot_serve_statistics* out) {
    if (!s || !out) return err(PILOT_EINVAL, "server and out must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->admitted = s->admitted;
    out->rejected = s->rejected;
    out->completed = s->completed;
    out->steps = s->steps;
    out->slots = s->slots;
    out->in_flight = int32_t(s->in_flight_requests());
    out->queued = int32_t(s->queue.size());
    int32_t ov = 0;   // read without waiting for the step in flight
    if (cudaMemcpy(&ov, s->vis_overflow, 4, cudaMemcpyDeviceToHost) == cudaSuccess) out->visited_overflows = ov;
    else cudaGetLastError();
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, size_t(p * double(l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : l) sum += x;
        out->mean_ms = sum / double(l.size());
        if (s->t_last_done > s->t_first_submit)
            out->qps = double(s->completed) / ((s->t_last_done - s->t_first_submit) / 1000.0);
    }
    return PILOT_OK;
}

void pilot_serve_destroy(pilot_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;   // synchronises the lanes' streams first
}

}  // extern "C"
