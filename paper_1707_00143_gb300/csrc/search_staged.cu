// search_staged.cu -- the search kernels with staged row gathers (each warp's
// rows of more than 512 values copied into a shared-memory ring by the bulk-
// copy engine, stage.cuh), pools in shared memory.
#include "search_kern.cuh"

namespace nsg {

cudaError_t launch_search_staged(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, int wpq,
                                 cudaStream_t st) {
    return launch_search_args<false, true>(a, l, per_warp, 0, false, wpq, st);
}

}  // namespace nsg
