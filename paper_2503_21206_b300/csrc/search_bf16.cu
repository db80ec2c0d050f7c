// search_bf16.cu -- the staged search kernels for BF16 reduced rows,
// both metrics (squared L2 and inner product).
#include "search_impl.cuh"

namespace pilot {

cudaError_t launch_search_dt1(const DevIndex& ix, const SearchConfig& cfg, const SearchIO& io, cudaStream_t st,
                               int num_sms) {
    return ix.metric == 0 ? launch_t<1, 0>(ix, cfg, io, st, num_sms) : launch_t<1, 1>(ix, cfg, io, st, num_sms);
}

cudaError_t prepare_serve_step_dt1(const DevIndex& ix, const SearchConfig& cfg, int num_sms, int max_warps,
                                    int* blocks, size_t* smem) {
    return ix.metric == 0 ? serve_prepare_t<1, 0>(ix, cfg, num_sms, max_warps, blocks, smem)
                          : serve_prepare_t<1, 1>(ix, cfg, num_sms, max_warps, blocks, smem);
}

cudaError_t launch_serve_step_dt1(const DevIndex& ix, const SearchConfig& cfg, const ServeIO& sio, cudaStream_t st,
                                   int blocks, size_t smem) {
    return ix.metric == 0 ? serve_launch_t<1, 0>(ix, cfg, sio, st, blocks, smem)
                          : serve_launch_t<1, 1>(ix, cfg, sio, st, blocks, smem);
}

}  // namespace pilot
