// search_global.cu -- the search kernels with each query's pool in a global-
// memory slot (pool sizes above what shared memory holds, or by choice).
#include "search_kern.cuh"

namespace nsg {

cudaError_t launch_search_global(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, size_t per_cta,
                                 bool stop, int wpq, cudaStream_t st) {
    return launch_search_args<true>(a, l, per_warp, per_cta, stop, wpq, st);
}

}  // namespace nsg
