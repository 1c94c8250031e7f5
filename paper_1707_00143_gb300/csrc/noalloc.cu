// noalloc.cu -- nsg_navigate_noalloc: the navigating-node search without any
// device allocation.
//
// Who needs it: callers that may not allocate device memory themselves --
// for instance code running inside a framework whose caching allocator has
// reserved (nearly) all of HBM, where a raw cudaMalloc fails or steals memory
// the framework accounts for, and latency-sensitive serving loops, where the
// device-wide synchronisation implied by cudaFree stalls every other stream.
// nsg_navigate allocates a visited bitmap of n bits per call; this variant
// uses a fixed bitmap in a file-scope __device__ array instead.
//
// That array is held by every GPU that loads this library, until the process
// exits: 2 MiB of bitmap (NSG_NOALLOC_MAX_N = 16,777,216 nodes) plus a few
// status words.  All calls on a device share it and it keeps the previous
// call's contents, so each call clears the part it uses first; two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <atomic>

#include <cuda_runtime.h>

#include "kernels.h"
#include "nsg.h"

namespace {

constexpr int64_t kMaxN = NSG_NOALLOC_MAX_N;
constexpr int64_t kWords = kMaxN / 32;
constexpr int kStatusWords = 4;  // [0] nav, [1] step-cap status, [2] bad-id flag

// visited bitmap followed by the status words
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords + kStatusWords];

constexpr int kMaxDevices = 64;
std::atomic<uint32_t *> g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up on the first
// call on that device (the host-side symbol is a stand-in, not a device
// address).  Two host threads making their first call at once both look it
// up and store the same address.  The cached address belongs to the device's
// current context: a cudaDeviceReset on that device invalidates it (as it
// does every index this library holds there).
cudaError_t scratch_ptr(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    uint32_t *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        void *v = nullptr;
        e = cudaGetSymbolAddress(&v, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        p = static_cast<uint32_t *>(v);
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

__global__ void noalloc_check_ids_kernel(const int *ids, int64_t count, int64_t n, uint32_t *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < count;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int v = ids[x];
        if (v < -1 || v >= n) atomicOr(bad, 1u);
    }
}

nsg_status fail(cudaError_t e) {
    nsg::record_cuda_error(e, "nsg_navigate_noalloc");
    return NSG_ECUDA;
}

}  // namespace

extern "C" nsg_status nsg_navigate_noalloc(const float *base_dev, int64_t n, int32_t d,
                                           const int32_t *knn_ids_dev, int32_t K, const double *centroid_dev,
                                           int32_t start, int32_t L, int32_t *nav_host, void *stream) {
    if (!base_dev || !knn_ids_dev || !centroid_dev || !nav_host || n < 1 || d < 1 ||
        d > 4 * nsg::MAX_DP4_HOST || K < 1 || L < 1 || L > 1024 || start < 0 || start >= n)
        return NSG_EINVAL;
    if (n > kMaxN) return NSG_EINVAL;  // beyond the fixed bitmap: use nsg_navigate
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *scratch = nullptr;
    cudaError_t e = scratch_ptr(&scratch);
    if (e != cudaSuccess) return fail(e);
    uint32_t *visited = scratch;
    uint32_t *status = scratch + kWords;
    const int64_t words = (n + 31) / 32;
    // the array keeps the previous call's contents: clear what this call uses
    if ((e = cudaMemsetAsync(status, 0, kStatusWords * sizeof(uint32_t), st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(visited, 0, words * sizeof(uint32_t), st)) != cudaSuccess) return fail(e);
    const int64_t count = n * (int64_t)K;
    int64_t blocks = (count + 255) / 256;
    const int64_t cap = (int64_t)nsg::sm_count() * 8;
    noalloc_check_ids_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(knn_ids_dev, count, n, status + 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    uint32_t h[kStatusWords] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    if (h[2]) return NSG_EINVAL;  // an id outside [-1, n): the gather would read out of range
    e = nsg::launch_navigate(base_dev, n, d, knn_ids_dev, K, centroid_dev, start, L, visited, nsg::default_steps(L),
                             reinterpret_cast<int *>(status), reinterpret_cast<int *>(status + 1), st);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    *nav_host = static_cast<int32_t>(h[0]);
    return h[1] ? NSG_ESTEPCAP : NSG_OK;
}
