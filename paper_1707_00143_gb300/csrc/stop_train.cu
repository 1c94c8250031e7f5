// stop_train.cu -- training of the learned early-termination rule on search
// traces, entirely on the GPU.
//
// A trace holds, for every expansion step t of a query, the state features
// seen before the step (search_core.cuh) and whether the step changed the
// first k pool entries.  The stop decision at step t is right exactly when
// no later step changes them, so the label of step t is
//     y_t = 1  iff  t > (last step that changed the first k entries).
// Model: z = w2 . relu(W1 f + b1) + b2, p = sigmoid(z), loss = mean binary
// cross-entropy over all steps of all queries; full-batch Adam.  FP32 master
// weights, FP16 export for the search kernel.
#include <cuda_fp16.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "search_core.cuh"

namespace nsg {

namespace {

constexpr int NP = NSG_STOP_PARAMS;
constexpr int NF = NSG_STOP_NF;
constexpr int NH = NSG_STOP_H;
// parameter offsets inside the flat vector
constexpr int OW1 = 0, OB1 = NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // SplitMix64 finaliser
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Glorot-uniform weights, zero biases.
__global__ void stop_init_kernel(float *w, uint64_t seed) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    float a = 0.0f;
    if (p < OB1) a = sqrtf(6.0f / (NF + NH));
    else if (p >= OW2 && p < OB2) a = sqrtf(6.0f / (NH + 1));
    const double u = (double)(mix64(seed * 0x100000001b3ULL + (uint64_t)p) >> 11) * (1.0 / 9007199254740992.0);
    w[p] = a * (float)(2.0 * u - 1.0);
}

// last[q] = last step that changed the first k entries (-1 if none); count = sum of trace lengths
__global__ void stop_last_kernel(const unsigned char *flag, const int *steps, int64_t nq, int cap, int *last,
                                 unsigned long long *count) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int T = steps[q] < cap ? steps[q] : cap;
        int l = -1;
        for (int t = T - 1; t >= 0; --t)
            if (flag[q * cap + t]) {
                l = t;
                break;
            }
        last[q] = l;
        atomicAdd(count, (unsigned long long)(T > 0 ? T : 0));
    }
}

// One warp per query: forward + backward over its steps, gradients kept in
// lane registers (lane owns hidden units lane and lane+32), then added to grad.
__global__ void __launch_bounds__(256) stop_grad_kernel(const float *feat, const int *steps, const int *last,
                                                       int64_t nq, int cap, const float *w, float *grad,
                                                       float *loss) {
    __shared__ float sw[NP];
    for (int p = threadIdx.x; p < NP; p += blockDim.x) sw[p] = w[p];
    __syncthreads();
    const unsigned lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float gw1[2][NF], gb1[2], gw2[2], gb2 = 0.0f, lsum = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        gb1[h] = gw2[h] = 0.0f;
#pragma unroll
        for (int i = 0; i < NF; ++i) gw1[h][i] = 0.0f;
    }
    for (int64_t q = warp; q < nq; q += nwarps) {
        const int T = steps[q] < cap ? steps[q] : cap;
        const int lq = last[q];
        for (int t = 0; t < T; ++t) {
            const float *fp = feat + ((int64_t)q * cap + t) * NF;
            float f[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) f[i] = __ldg(fp + i);
            const float y = t > lq ? 1.0f : 0.0f;
            float a[2], part = 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                float s = sw[OB1 + j];
#pragma unroll
                for (int i = 0; i < NF; ++i) s = fmaf(sw[OW1 + j * NF + i], f[i], s);
                a[h] = s;
                part = fmaf(sw[OW2 + j], fmaxf(s, 0.0f), part);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(NSG_FULL, part, o);
            const float z = part + sw[OB2];
            const float p = 1.0f / (1.0f + __expf(-z));
            // BCE with logits: log(1 + e^z) - y z, computed stably
            lsum += fmaxf(z, 0.0f) - y * z + log1pf(__expf(-fabsf(z)));
            const float dz = p - y;
            gb2 += dz;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                const float hj = fmaxf(a[h], 0.0f);
                gw2[h] = fmaf(dz, hj, gw2[h]);
                const float dh = a[h] > 0.0f ? dz * sw[OW2 + j] : 0.0f;
                gb1[h] += dh;
#pragma unroll
                for (int i = 0; i < NF; ++i) gw1[h][i] = fmaf(dh, f[i], gw1[h][i]);
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        atomicAdd(grad + OB1 + j, gb1[h]);
        atomicAdd(grad + OW2 + j, gw2[h]);
#pragma unroll
        for (int i = 0; i < NF; ++i) atomicAdd(grad + OW1 + j * NF + i, gw1[h][i]);
    }
    if (lane == 0) {
        atomicAdd(grad + OB2, gb2);
        if (loss) atomicAdd(loss, lsum);
    }
}

// Adam step on the mean gradient; clears the gradient; writes the FP16 export.
__global__ void stop_adam_kernel(float *w, float *grad, float *m, float *v, const unsigned long long *count,
                                 int step, float lr, __half *out, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const float inv = 1.0f / (float)(*count > 0 ? *count : 1);
    if (p == 0 && loss) *loss *= inv;  // one sum per warp was added: mean over samples
    if (p >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[p] * inv;
    grad[p] = 0.0f;
    m[p] = b1 * m[p] + (1.0f - b1) * g;
    v[p] = b2 * v[p] + (1.0f - b2) * g * g;
    const float mh = m[p] / (1.0f - powf(b1, (float)step));
    const float vh = v[p] / (1.0f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + eps);
    out[p] = __float2half_rn(w[p]);
}

}  // namespace

cudaError_t run_stop_train(const float *feat, const unsigned char *flag, const int *steps, int64_t nq, int cap,
                           int iters, float lr, uint64_t seed, float *master, void *model_out, float *loss_out,
                           cudaStream_t st) {
    float *scratch = nullptr;  // grad, m, v
    int *last = nullptr;
    unsigned long long *count = nullptr;
    cudaError_t e = cudaMalloc(&scratch, 3 * NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&last, (nq > 0 ? nq : 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&count, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, 3 * NP * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && loss_out) e = cudaMemsetAsync(loss_out, 0, iters * sizeof(float), st);
    if (e == cudaSuccess && seed != 0) {
        stop_init_kernel<<<(NP + 255) / 256, 256, 0, st>>>(master, seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t blocks = (nq + 255) / 256;
        stop_last_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(flag, steps, nq, cap, last, count);
        e = cudaGetLastError();
    }
    const int64_t gblocks = (nq + 7) / 8;  // 8 warps per block, one query per warp
    const int grid = (int)(gblocks < (int64_t)sm_count() * 8 ? gblocks : (int64_t)sm_count() * 8);
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
        float *lp = loss_out ? loss_out + it : nullptr;
        stop_grad_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(feat, steps, last, nq, cap, master, scratch, lp);
        stop_adam_kernel<<<(NP + 255) / 256, 256, 0, st>>>(master, scratch, scratch + NP, scratch + 2 * NP, count,
                                                          it + 1, lr, reinterpret_cast<__half *>(model_out), lp);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    cudaFree(scratch);
    cudaFree(last);
    cudaFree(count);
    return e;
}

}  // namespace nsg
