// knn.cu -- exact k nearest neighbours by serial scan (Section 4.1.2 item 1),
// FP32 on CUDA cores.  It is the kNN-graph initialisation of Alg. 2 (self
// join, own id skipped) and the ground truth of the precision metric (Eq. 1).
//
// One CTA = 8 warps x 4 queries.  Base rows stream through shared memory in
// tiles of 128 rows (d in chunks of 128 floats, row stride +4 floats so the
// 16-byte reads of 8 lanes hit 32 distinct banks).  Lane l owns rows
// l, l+32, l+64, l+96 of a tile for its warp's 4 queries (16 accumulators).
// After each tile a query's new keys below its current k-th key are merged
// into its sorted top-k list in shared memory (warp_merge).
#include "common.cuh"
#include "kernels.h"
#include "search_core.cuh"

namespace nsg {

constexpr int KD_TB = 128;  // base rows per tile
constexpr int KD_DC = 128;  // floats per d-chunk
constexpr int KD_WARPS = 8;
constexpr int KD_QPW = 4;
constexpr int KD_QPB = KD_WARPS * KD_QPW;
constexpr int KD_MAXK = 256;

struct KnnArgs {
    const float4 *base4;
    int64_t n;
    int dp4;
    const float *queries;  // [nq][dp]
    int64_t nq, q0;
    int k, self_join;
    int *ids;
    float *d2;
};

static size_t knn_smem_bytes(int k) {
    return 4ull * KD_TB * (KD_DC + 4) + 16ull * KD_WARPS * KD_DC + 8ull * KD_QPB * k +
           3ull * 8 * KD_WARPS * KD_TB + 2ull * 4 * KD_WARPS * KD_TB;
}

template <int E>
__device__ __forceinline__ float comp(const float4 &v) {
    return E == 0 ? v.x : E == 1 ? v.y : E == 2 ? v.z : v.w;
}

__global__ void __launch_bounds__(256, 1) knn_direct_kernel(KnnArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *bt = reinterpret_cast<float *>(smem);
    float4 *qs = reinterpret_cast<float4 *>(bt + KD_TB * (KD_DC + 4));
    uint64_t *lists = reinterpret_cast<uint64_t *>(qs + KD_WARPS * KD_DC);
    uint64_t *cbuf = lists + (size_t)KD_QPB * a.k;
    uint64_t *ck = cbuf + KD_WARPS * KD_TB;
    uint64_t *sk = ck + KD_WARPS * KD_TB;
    int *cp = reinterpret_cast<int *>(sk + KD_WARPS * KD_TB);
    int *sp = cp + KD_WARPS * KD_TB;
    __shared__ int sizes[KD_QPB];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t qbase = (int64_t)blockIdx.x * KD_QPB;
    const int dp = a.dp4 * 4;
    if (tid < KD_QPB) sizes[tid] = 0;
    uint64_t *wc = cbuf + warp * KD_TB, *wck = ck + warp * KD_TB, *wsk = sk + warp * KD_TB;
    int *wcp = cp + warp * KD_TB, *wsp = sp + warp * KD_TB;

    for (int64_t t0 = 0; t0 < a.n; t0 += KD_TB) {
        float acc[4][KD_QPW];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < KD_QPW; ++q) acc[r][q] = 0.0f;
        for (int c0 = 0; c0 < dp; c0 += KD_DC) {
            const int dc = dp - c0 < KD_DC ? dp - c0 : KD_DC;  // multiple of 4
            const int dc4 = dc >> 2;
            __syncthreads();
            for (int x = tid; x < KD_TB * dc4; x += blockDim.x) {
                int r = x / dc4, c4 = x - r * dc4;
                int64_t row = t0 + r;
                float4 v = row < a.n ? __ldg(a.base4 + row * a.dp4 + (c0 >> 2) + c4)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                *reinterpret_cast<float4 *>(bt + r * (KD_DC + 4) + c4 * 4) = v;
            }
            for (int x = tid; x < KD_QPB * dc; x += blockDim.x) {
                int qi = x / dc, kk = x - qi * dc;
                int64_t qg = qbase + qi;
                float v = qg < a.nq ? __ldg(a.queries + qg * dp + c0 + kk) : 0.0f;
                reinterpret_cast<float *>(qs)[((qi / KD_QPW) * KD_DC + kk) * 4 + (qi % KD_QPW)] = v;
            }
            __syncthreads();
            const float4 *qw = qs + warp * KD_DC;
            for (int kk = 0; kk < dc; kk += 4) {
                float4 b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    b[r] = *reinterpret_cast<const float4 *>(bt + (lane + 32 * r) * (KD_DC + 4) + kk);
#define NSG_KD_STEP(E)                                                      \
    {                                                                       \
        const float4 q = qw[kk + E];                                        \
        _Pragma("unroll") for (int r = 0; r < 4; ++r) {                     \
            const float be = comp<E>(b[r]);                                 \
            float t0_ = be - q.x, t1_ = be - q.y, t2_ = be - q.z, t3_ = be - q.w; \
            acc[r][0] += t0_ * t0_;                                         \
            acc[r][1] += t1_ * t1_;                                         \
            acc[r][2] += t2_ * t2_;                                         \
            acc[r][3] += t3_ * t3_;                                         \
        }                                                                   \
    }
                NSG_KD_STEP(0)
                NSG_KD_STEP(1)
                NSG_KD_STEP(2)
                NSG_KD_STEP(3)
#undef NSG_KD_STEP
            }
        }
        // selection: keys below the query's current k-th key join its list
#pragma unroll
        for (int qi = 0; qi < KD_QPW; ++qi) {
            const int ql = warp * KD_QPW + qi;
            const int64_t qg = qbase + ql;
            if (qg >= a.nq) continue;
            uint64_t *list = lists + (size_t)ql * a.k;
            int size = sizes[ql];
            const uint64_t tail = size >= a.k ? kval(list[a.k - 1]) : ~0ull;
            int m = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t id = t0 + lane + 32 * r;
                const uint64_t key = make_key(acc[r][qi], (int)id);
                const bool keep = id < a.n && !(a.self_join && id == a.q0 + qg) && key < tail;
                const unsigned bal = __ballot_sync(NSG_FULL, keep);
                if (keep) wc[m + __popc(bal & lanemask_lt())] = key;
                m += __popc(bal);
            }
            __syncwarp();
            if (m > 0) {
                warp_merge(list, a.k, size, wc, m, wck, wcp, wsk, wsp);
                if (lane == 0) sizes[ql] = size;
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int qi = 0; qi < KD_QPW; ++qi) {
        const int ql = warp * KD_QPW + qi;
        const int64_t qg = qbase + ql;
        if (qg >= a.nq) continue;
        const uint64_t *list = lists + (size_t)ql * a.k;
        const int size = sizes[ql];
        for (int t = lane; t < a.k; t += 32) {
            a.ids[qg * a.k + t] = t < size ? kid(list[t]) : -1;
            if (a.d2) a.d2[qg * a.k + t] = t < size ? kd2(list[t]) : __int_as_float(0x7f800000);
        }
    }
}

cudaError_t launch_knn_direct(const KnnLaunch &l, cudaStream_t st) {
    if (l.nq <= 0) return cudaSuccess;
    if (l.k > KD_MAXK || (l.dp & 3)) return cudaErrorInvalidValue;
    KnnArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.n = l.n;
    a.dp4 = l.dp / 4;
    a.queries = l.queries;
    a.nq = l.nq;
    a.q0 = l.q0;
    a.k = l.k;
    a.self_join = l.self_join;
    a.ids = l.ids;
    a.d2 = l.d2;
    size_t smem = knn_smem_bytes(l.k);
    cudaError_t e = cudaFuncSetAttribute(knn_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (l.nq + KD_QPB - 1) / KD_QPB;
    knn_direct_kernel<<<(unsigned)grid, KD_WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace nsg

// ---------------------------------------------------------------------------
// Exact re-rank of tensor-core candidates (float data): warp per query; the
// candidates' FP32 distances come from the same row-distance routine as the
// search, and the k smallest keys are kept with warp_merge.
// ---------------------------------------------------------------------------
namespace nsg {

struct RerankArgs {
    const float4 *base4;
    int dp4;
    const float *queries;  // [nq][dp] (self join: base rows q0..)
    int64_t nq;
    const int *cand;
    int KL, k;
    int *ids;
    float *d2;
};

template <int G, int V, int U>
__global__ void __launch_bounds__(256) knn_rerank_kernel(RerankArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    const size_t per = 8ull * (32 + a.k + 64) + 4ull * (32 + 64);
    unsigned char *base = smem + warp * ((per + 15) & ~size_t(15));
    uint64_t *keys = reinterpret_cast<uint64_t *>(base);
    uint64_t *list = keys + 32;
    uint64_t *ck = list + a.k, *sk = ck + 32;
    int *ids = reinterpret_cast<int *>(sk + 32);
    int *cp = ids + 32, *sp = cp + 32;
    for (int64_t q = (int64_t)blockIdx.x * wpb + warp; q < a.nq; q += (int64_t)gridDim.x * wpb) {
        RowQuery<G, V> Q;
        Q.load_row(reinterpret_cast<const float4 *>(a.queries) + q * a.dp4, a.dp4);
        int size = 0;
        for (int c0 = 0; c0 < a.KL; c0 += 32) {
            const int c = c0 + (int)lane;
            const int id = c < a.KL ? a.cand[q * a.KL + c] : -1;
            const unsigned bal = __ballot_sync(NSG_FULL, id >= 0);
            if (id >= 0) ids[__popc(bal & lanemask_lt())] = id;
            const int m = __popc(bal);
            __syncwarp();
            if (m == 0) break;
            rows_dist<G, V, U>(Q, a.base4, a.dp4, ids, m, keys);
            warp_merge(list, a.k, size, keys, m, ck, cp, sk, sp);
        }
        for (int t = lane; t < a.k; t += 32) {
            a.ids[q * a.k + t] = t < size ? kid(list[t]) : -1;
            if (a.d2) a.d2[q * a.k + t] = t < size ? kd2(list[t]) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

cudaError_t launch_knn_rerank(const KnnLaunch &l, const int *cand, int KL, cudaStream_t st) {
    RerankArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.dp4 = l.dp / 4;
    a.queries = l.self_join ? l.base + l.q0 * l.dp : l.queries;
    a.nq = l.nq;
    a.cand = cand;
    a.KL = KL;
    a.k = l.k;
    a.ids = l.ids;
    a.d2 = l.d2;
    const int wpb = 8;
    const size_t per = ((8ull * (32 + l.k + 64) + 4ull * (32 + 64)) + 15) & ~size_t(15);
    const size_t smem = per * wpb;
    const int64_t blocks = (l.nq + wpb - 1) / wpb;
    const int grid = (int)(blocks < (int64_t)sm_count() * 16 ? blocks : (int64_t)sm_count() * 16);
    cudaError_t e = cudaSuccess;
    NSG_DISPATCH_DP4(a.dp4, {
        auto kern = knn_rerank_kernel<G_, V_, U_>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            kern<<<grid, wpb * 32, smem, st>>>(a);
            e = cudaGetLastError();
        }
    });
    return e;
}

}  // namespace nsg
