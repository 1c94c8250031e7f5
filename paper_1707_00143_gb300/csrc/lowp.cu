// lowp.cu -- building the BF16 / FP8-e4m3 / U8 copies of the base used by
// the precision forms of the search.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"

namespace nsg {

bool make_gather_map(void *map, const void *rows, int64_t n, int row_bytes) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return false;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    if (row_bytes <= 0 || row_bytes % 16 || row_bytes > 2048 || n < 1 || n > INT32_MAX) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / 8), (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / 8), 1};  // one whole row, one row high
    cuuint32_t estr[2] = {1, 1};
    return fn(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(rows), dims,
              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__global__ void absmax_kernel(const float *__restrict__ x, int64_t count, unsigned *out) {
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(NSG_FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_absmax(const float *x, int64_t count, unsigned *out_bits, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    absmax_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(x, count, out_bits);
    return cudaGetLastError();
}

__device__ __forceinline__ unsigned order_key(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void minmax_kernel(const float *__restrict__ x, int64_t n, int dp, int d, unsigned *out) {
    unsigned lo = 0xffffffffu, hi = 0u;
    bool frac = false;
    const int64_t total = n * d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[(i / d) * dp + i % d];
        const unsigned kk = order_key(v);
        lo = min(lo, kk);
        hi = max(hi, kk);
        frac |= rintf(v) != v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(NSG_FULL, lo, o));
        hi = max(hi, __shfl_xor_sync(NSG_FULL, hi, o));
    }
    const bool any_frac = __any_sync(NSG_FULL, frac);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
        if (any_frac) atomicOr(out + 2, 1u);
    }
}

cudaError_t launch_minmax(const float *x, int64_t n, int dp, int d, unsigned *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n * d + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    minmax_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(x, n, dp, d, out);
    return cudaGetLastError();
}

template <int P>
__global__ void to_lowp_kernel(const float *__restrict__ src, int64_t n, int dp, int d, float scale, float lo,
                               void *dst, int dpl, int *inexact) {
    const int64_t total = n * dpl;
    bool bad = false;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = x / dpl;
        const int c = (int)(x % dpl);
        const float v = c < d ? src[r * dp + c] : 0.0f;
        if (P == 1) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            reinterpret_cast<__nv_bfloat16 *>(dst)[x] = h;
            bad |= __bfloat162float(h) != v;
        } else if (P == 3) {
            const float y = (v - lo) * scale;
            const float u = c < d ? fminf(fmaxf(rintf(y), 0.0f), 255.0f) : 0.0f;
            reinterpret_cast<unsigned char *>(dst)[x] = (unsigned char)u;
            bad |= c < d && u != y;
        } else {
            const __nv_fp8_storage_t h = __nv_cvt_float_to_fp8(v * scale, __NV_SATFINITE, __NV_E4M3);
            reinterpret_cast<__nv_fp8_storage_t *>(dst)[x] = h;
            const __half_raw hr = __nv_cvt_fp8_to_halfraw(h, __NV_E4M3);
            bad |= __half2float(*reinterpret_cast<const __half *>(&hr)) != v * scale;
        }
    }
    if (__any_sync(NSG_FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(inexact, 1);
}

cudaError_t launch_to_lowp(const float *src, int64_t n, int dp, int d, int precision, float scale, float lo,
                           void *dst, int dpl, int *inexact, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n * dpl + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 16;
    const int g = (int)(blocks < cap ? blocks : cap);
    if (precision == 1) to_lowp_kernel<1><<<g, 256, 0, st>>>(src, n, dp, d, scale, lo, dst, dpl, inexact);
    else if (precision == 2) to_lowp_kernel<2><<<g, 256, 0, st>>>(src, n, dp, d, scale, lo, dst, dpl, inexact);
    else to_lowp_kernel<3><<<g, 256, 0, st>>>(src, n, dp, d, scale, lo, dst, dpl, inexact);
    return cudaGetLastError();
}

}  // namespace nsg
