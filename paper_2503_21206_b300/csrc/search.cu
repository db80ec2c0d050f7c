// search.cu -- host side of the staged search: launch-shape defaults, the
// visited-table size, and the dispatch to the kernels of each reduced-row
// type (search_f32.cu, search_bf16.cu, search_fp8.cu; the kernels themselves
// are in search_impl.cuh).
#include "search_impl.cuh"

namespace pilot {

size_t serve_smem_per_block(const DevIndex& ix, const SearchConfig& cfg) {
    return make_layout(ix, cfg).per_warp * size_t(cfg.warps_per_block);
}

cudaError_t prepare_serve_step(const DevIndex& ix, const SearchConfig& cfg, int num_sms, int max_warps, int* blocks,
                               size_t* smem) {
    switch (ix.red_dtype) {
        case 0: return prepare_serve_step_dt0(ix, cfg, num_sms, max_warps, blocks, smem);
        case 1: return prepare_serve_step_dt1(ix, cfg, num_sms, max_warps, blocks, smem);
        case 2: return prepare_serve_step_dt2(ix, cfg, num_sms, max_warps, blocks, smem);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_serve_step(const DevIndex& ix, const SearchConfig& cfg, const ServeIO& sio, cudaStream_t st,
                              int blocks, size_t smem) {
    switch (ix.red_dtype) {
        case 0: return launch_serve_step_dt0(ix, cfg, sio, st, blocks, smem);
        case 1: return launch_serve_step_dt1(ix, cfg, sio, st, blocks, smem);
        case 2: return launch_serve_step_dt2(ix, cfg, sio, st, blocks, smem);
        default: return cudaErrorInvalidValue;
    }
}

size_t search_smem_per_warp(const DevIndex& ix, const SearchConfig& cfg) { return make_layout(ix, cfg).per_warp; }

SearchConfig default_search_config(const DevIndex& ix, int k, int ef) {
    SearchConfig cfg{};
    cfg.k = k;
    cfg.ef = ef;
    cfg.stage1 = 1;
    cfg.stage2_expansions = 2;
    cfg.stage3 = 1;
    cfg.use_fes = 1;
    cfg.fes_T = kFesT;
    cfg.fes_seeds = 1;
    cfg.warps_per_block = 2;
    // 24 rows of the widest kind per gather pass (an expansion probes its
    // neighbours first and gathers only the unvisited ones, typically fewer
    // than 24 of 32), at most ~16.5 KB, in whole groups of 4 rows (the
    // pre-filter's eight-lanes-per-row layout takes 4 rows at a time), at
    // least 4 rows
    const int fs = stage_stride(ix.full_row_bytes), rs = stage_stride(ix.red_row_bytes);
    int full_rows = 16896 / fs;
    full_rows = full_rows > 24 ? 24 : (full_rows & ~3);
    if (full_rows < 4) full_rows = 4;
    const int stage = full_rows * (fs > rs ? fs : rs);
    // stage (1) copies all 32 neighbours' reduced rows during the probe when
    // they fit in this buffer; wider reduced rows are gathered after the
    // probe, like full rows, rather than enlarge it and cost occupancy
    cfg.stage_bytes = stage;
    cfg.filter = 1;
    set_visited_size(ix, cfg, ix.vis_stride);
    return cfg;
}

void set_visited_size(const DevIndex& ix, SearchConfig& cfg, int64_t entries_per_slot) {
    const VisSize v = vis_size_for(cfg.ef, ix.R > ix.R_sub ? ix.R : ix.R_sub, ix.id_bits, entries_per_slot);
    cfg.vis_mask = v.mask;
    cfg.vis_qbits = v.qbits;
}

void set_stage_rows(const DevIndex& ix, SearchConfig& cfg, int rows) {
    // rows of the widest row kind staged per pass (a multiple of 4, 4..32)
    rows = rows < 4 ? 4 : (rows > 32 ? 32 : rows & ~3);
    const int fs = stage_stride(ix.full_row_bytes), rs = stage_stride(ix.red_row_bytes);
    int stage = rows * (fs > rs ? fs : rs);
    cfg.stage_bytes = stage;
}

cudaError_t launch_search(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st,
                          int num_sms) {
    if (io.nq == 0) return cudaSuccess;
    switch (ix.red_dtype) {
        case 0: return launch_search_dt0(ix, cfg, io, st, num_sms);
        case 1: return launch_search_dt1(ix, cfg, io, st, num_sms);
        case 2: return launch_search_dt2(ix, cfg, io, st, num_sms);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pilot
