// search_staged_global.cu -- the staged-gather search kernels (stage.cuh)
// with each query's pool in a global-memory slot.
#include "search_kern.cuh"

namespace nsg {

cudaError_t launch_search_staged_global(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, int wpq,
                                        cudaStream_t st) {
    return launch_search_args<true, true>(a, l, per_warp, 0, false, wpq, st);
}

}  // namespace nsg
