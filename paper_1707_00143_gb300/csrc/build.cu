// build.cu -- Alg. 2 kernels other than the per-node search: centroid,
// navigating node, MRNG edge selection, reachability BFS helpers of the
// connectivity pass (the pass itself is in connect.cu); plus the
// precision count (Eq. 1) and a row-padding copy.
#include <climits>

#include "kernels.h"
#include "search_core.cuh"

namespace nsg {

__host__ __device__ static inline int round32(int x) { return (x + 31) & ~31; }
static inline int log2i(unsigned x) {
    int r = 0;
    while ((1u << r) < x) ++r;
    return r;
}

template <typename T>
__device__ __forceinline__ T ld_volatile(const T *p) {
    return *reinterpret_cast<const volatile T *>(p);
}

// ---------------------------------------------------------------------------
// Centroid (Alg. 2, first step): block b sums rows [b*rows, (b+1)*rows) of every
// column in FP64 (row order), then one pass adds the block sums in block order
// and divides by n.  On integer data every partial sum is exact.
// ---------------------------------------------------------------------------
__global__ void centroid_partial_kernel(const float *__restrict__ base, int64_t n, int d,
                                        int64_t rows, double *__restrict__ partial) {
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = r0 + rows < n ? r0 + rows : n;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s = __dadd_rn(s, (double)__ldg(base + r * d + j));
        partial[(int64_t)blockIdx.x * d + j] = s;
    }
}

__global__ void centroid_final_kernel(const double *__restrict__ partial, int nb, int d, int64_t n,
                                      double *__restrict__ c) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s = __dadd_rn(s, partial[(int64_t)b * d + j]);
        c[j] = __ddiv_rn(s, (double)n);
    }
}

cudaError_t launch_centroid(const float *base, int64_t n, int d, double *partial, int nblocks,
                            double *c, cudaStream_t st) {
    int64_t rows = (n + nblocks - 1) / nblocks;
    int nb = (int)((n + rows - 1) / rows);
    int threads = d < 256 ? round32(d) : 256;
    centroid_partial_kernel<<<nb, threads, 0, st>>>(base, n, d, rows, partial);
    centroid_final_kernel<<<(d + 255) / 256, 256, 0, st>>>(partial, nb, d, n, c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Navigating node (Alg. 2; Section 3.5 ii): Alg. 1 on the kNN graph from `start`
// toward the centroid, one warp.  Distances are FP64 sums over j in order with
// explicitly rounded operations (no FMA), so they do not depend on the
// compiler.  Lanes compute the distances of the new neighbours; lane 0 keeps
// the sorted pool (one query: simplicity over speed).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool dkey_less(double da, int ia, double db, int ib) {
    return da < db || (da == db && ia < ib);
}

__global__ void navigate_kernel(const float *__restrict__ base, int d, const int *__restrict__ knn,
                                int K, const double *__restrict__ cg, int start, int L,
                                uint32_t *visited, int max_steps, int *nav_out, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Wk = round32(K);
    double *c = reinterpret_cast<double *>(smem);
    double *pd = c + d;
    double *cd = pd + (L + 1);
    int *pid = reinterpret_cast<int *>(cd + Wk);
    int *pchk = pid + (L + 1);
    int *cid = pchk + (L + 1);
    const unsigned lane = threadIdx.x & 31;
    for (int j = lane; j < d; j += 32) c[j] = cg[j];
    __syncwarp();
    auto dist = [&](int id) -> double {
        const float *x = base + (int64_t)id * d;
        double s = 0.0;
        for (int j = 0; j < d; ++j) {
            double t = __dsub_rn((double)__ldg(x + j), c[j]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        return s;
    };
    int size = 1;
    if (lane == 0) {
        atomicOr(visited + (start >> 5), 1u << (start & 31));
        pd[0] = dist(start);
        pid[0] = start;
        pchk[0] = 0;
    }
    __syncwarp();
    int steps = 0;
    bool capped = false;
    for (;;) {
        int i = -1;
        if (lane == 0)
            for (int t = 0; t < size; ++t)
                if (!pchk[t]) {
                    i = t;
                    break;
                }
        i = __shfl_sync(NSG_FULL, i, 0);
        if (i < 0) break;
        if (steps >= max_steps) {
            capped = true;
            break;
        }
        ++steps;
        if (lane == 0) pchk[i] = 1;
        __syncwarp();
        const int u = pid[i];
        int m = 0;
        for (int b = 0; b < K; b += 32) {
            int slot = b + lane;
            int w = slot < K ? __ldg(knn + (int64_t)u * K + slot) : -1;
            bool fresh = false;
            if (w >= 0) {
                uint32_t bit = 1u << (w & 31);
                fresh = !(atomicOr(visited + (w >> 5), bit) & bit);
            }
            unsigned bal = __ballot_sync(NSG_FULL, fresh);
            if (fresh) cid[m + __popc(bal & lanemask_lt())] = w;
            m += __popc(bal);
        }
        __syncwarp();
        for (int t = lane; t < m; t += 32) cd[t] = dist(cid[t]);
        __syncwarp();
        if (lane == 0) {
            for (int t = 0; t < m; ++t) {
                double dv = cd[t];
                int iv = cid[t];
                if (size == L && !dkey_less(dv, iv, pd[L - 1], pid[L - 1])) continue;
                int pos = size < L ? size : L - 1;
                while (pos > 0 && dkey_less(dv, iv, pd[pos - 1], pid[pos - 1])) {
                    pd[pos] = pd[pos - 1];
                    pid[pos] = pid[pos - 1];
                    pchk[pos] = pchk[pos - 1];
                    --pos;
                }
                pd[pos] = dv;
                pid[pos] = iv;
                pchk[pos] = 0;
                if (size < L) ++size;
            }
        }
        size = __shfl_sync(NSG_FULL, size, 0);
        __syncwarp();
    }
    if (lane == 0) {
        *nav_out = pid[0];
        *status = capped ? -4 : 0;
    }
}

cudaError_t launch_navigate(const float *base, int64_t n, int d, const int *knn, int K,
                            const double *c, int start, int L, uint32_t *visited_bits,
                            int max_steps, int *nav_out, int *status, cudaStream_t st) {
    (void)n;
    int Wk = round32(K);
    size_t smem = 8ull * (d + (L + 1) + Wk) + 4ull * (2 * (L + 1) + Wk);
    cudaError_t e = cudaFuncSetAttribute(navigate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    navigate_kernel<<<1, 32, smem, st>>>(base, d, knn, K, c, start, L, visited_bits, max_steps,
                                         nav_out, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MRNG edge selection (Alg. 2; Section 3.3), one warp per node.  Candidates are
// already sorted by key; the first is kept; a later candidate p is occluded
// when d2(p, r) < d2(p, v) for a kept r (r in the open lune of vp); stop at R.
//
// The warp takes the candidates in batches of NB = (32 / G) * B: each G-lane
// group holds B candidate rows in registers (batch position b * (32/G) + grp).
// The kept rows are read once per batch, U at a time, and every group measures
// them against its B candidates; the pass ends early once every candidate of
// the batch is occluded.  The survivors are then taken in candidate order:
// the first is kept, and the later survivors are measured against it (the
// kept set a sequential scan would have at their turn), and so on.  Results,
// and the count of candidates examined, equal the one-at-a-time scan.
// ---------------------------------------------------------------------------
struct PruneArgs {
    const float4 *base4;
    int dp4;
    const int *cand_ids;
    const float *cand_d2;
    const int *cand_count;
    int C, R, Wr;
    int64_t v0, nv;
    int *adj, *deg;
    unsigned long long *examined;
};

// Batch positions (b * P + g) whose flag is set in group g's lane 0, as a mask.
template <int G, int B>
__device__ __forceinline__ unsigned batch_mask(const bool (&f)[B]) {
    constexpr int P = 32 / G;
    const bool lead = lane_id() % G == 0;
    unsigned m = 0;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const unsigned bal = __ballot_sync(NSG_FULL, lead && f[b]);
#pragma unroll
        for (int g = 0; g < P; ++g) m |= ((bal >> (g * G)) & 1u) << (b * P + g);
    }
    return m;
}

template <int G, int V, int U, int B>
__device__ __forceinline__ void prune_body(const PruneArgs &a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int P = 32 / G, NB = P * B;
    static_assert(NB <= 32, "batch mask holds 32 positions");
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int lane = (int)lane_id(), grp = lane / G, sub = lane % G;
    int *kept = reinterpret_cast<int *>(smem) + (size_t)warp * a.Wr;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    unsigned long long examined = 0;
    for (int64_t j = (int64_t)blockIdx.x * wpb + warp; j < a.nv; j += stride) {
        const int64_t v = a.v0 + j;
        const int *ci = a.cand_ids + j * a.C;
        const float *cd = a.cand_d2 + j * a.C;
        int cnt = a.cand_count != nullptr ? min(max(a.cand_count[j], 0), a.C) : a.C;
        if (cnt > 0 && ci[0] < 0) cnt = 0;  // a negative id ends the list
        int nk = 0, t = 0;                  // kept; candidates examined
        if (cnt > 0) {
            if (lane == 0) kept[0] = ci[0];
            nk = 1;
            t = 1;
        }
        __syncwarp();
        while (t < cnt && nk < a.R) {
            float4 q[B][V];
            float pdv[B];
            bool occ[B];
            int id[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int c = t + b * P + grp;
                id[b] = c < cnt ? ci[c] : 0;
                occ[b] = id[b] < 0;
            }
            const unsigned neg = batch_mask<G, B>(occ);
            if (neg) cnt = t + __ffs(neg) - 1;  // a negative id ends the list
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int c = t + b * P + grp;
                const bool valid = c < cnt;
                pdv[b] = valid ? cd[c] : 0.0f;
                occ[b] = !valid;
                const float4 *row = a.base4 + (int64_t)(valid ? id[b] : 0) * a.dp4;
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    const int k = u * G + sub;
                    q[b][u] = (valid && k < a.dp4) ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            // against the kept set as it was before the batch
            for (int i0 = 0; i0 < nk; i0 += U) {
                bool all = true;
#pragma unroll
                for (int b = 0; b < B; ++b) all &= occ[b];
                if (__all_sync(NSG_FULL, all)) break;
                float4 x[U][V];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int i = i0 + u;
                    const float4 *row = a.base4 + (int64_t)(i < nk ? kept[i] : 0) * a.dp4;
#pragma unroll
                    for (int w = 0; w < V; ++w) {
                        const int k = w * G + sub;
                        x[u][w] = (i < nk && k < a.dp4) ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int b = 0; b < B; ++b) {
                        float s = 0.0f;
#pragma unroll
                        for (int w = 0; w < V; ++w) s += sq4(x[u][w], q[b][w]);
                        s = group_sum<G>(s);
                        if (i0 + u < nk && s < pdv[b]) occ[b] = true;
                    }
            }
            // survivors in candidate order, each measured against the ones kept before it
            bool live_f[B];
#pragma unroll
            for (int b = 0; b < B; ++b) live_f[b] = !occ[b];
            unsigned live = batch_mask<G, B>(live_f);
            int stop = -1;
            while (live) {
                const int pos = __ffs(live) - 1;
                live &= live - 1u;
                const int pj = ci[t + pos];
                if (lane == 0) kept[nk] = pj;
                ++nk;
                if (nk == a.R) {
                    stop = pos;
                    break;
                }
                if (!live) break;
                const float4 *row = a.base4 + (int64_t)pj * a.dp4;
                float4 x[V];
#pragma unroll
                for (int w = 0; w < V; ++w) {
                    const int k = w * G + sub;
                    x[w] = k < a.dp4 ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                bool hit[B];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    float s = 0.0f;
#pragma unroll
                    for (int w = 0; w < V; ++w) s += sq4(x[w], q[b][w]);
                    s = group_sum<G>(s);
                    hit[b] = s < pdv[b];
                }
                live &= ~batch_mask<G, B>(hit);
            }
            __syncwarp();
            t = stop >= 0 ? t + stop + 1 : min(t + NB, cnt);
        }
        examined += (unsigned long long)t;
        for (int e = lane; e < a.R; e += 32) a.adj[v * a.R + e] = e < nk ? kept[e] : -1;
        if (lane == 0) a.deg[v] = nk;
        __syncwarp();
    }
    if (a.examined != nullptr && lane == 0 && examined) atomicAdd(a.examined, examined);
}

// Rows of up to 4 float4s per lane run 3 blocks per SM (78 registers, no
// spills; 8 % faster than 2 blocks on 128-value rows); wider rows keep the
// compiler's own budget (at 3 blocks they spill and run 1.8x slower).
template <int G, int V, int U, int B>
__global__ void __launch_bounds__(256) prune_kernel(PruneArgs a) {
    prune_body<G, V, U, B>(a);
}
template <int G, int V, int U, int B>
__global__ void __launch_bounds__(256, 3) prune_narrow_kernel(PruneArgs a) {
    prune_body<G, V, U, B>(a);
}
template <int G, int V, int U, int B>
constexpr auto prune_entry() {
    if constexpr (V <= 4) return prune_narrow_kernel<G, V, U, B>;
    else return prune_kernel<G, V, U, B>;
}

// Candidate rows held per lane group: two while they fit in 32 float4s.
template <int V>
struct PruneBatch {
    static constexpr int value = V <= 8 ? 2 : 1;
};

cudaError_t launch_prune(const PruneLaunch &l, cudaStream_t st) {
    if (l.nv <= 0) return cudaSuccess;
    PruneArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.dp4 = l.dp / 4;
    a.cand_ids = l.cand_ids;
    a.cand_d2 = l.cand_d2;
    a.cand_count = l.cand_count;
    a.C = l.C;
    a.R = l.R;
    a.Wr = round32(l.R);
    a.v0 = l.v0;
    a.nv = l.nv;
    a.adj = l.adj;
    a.deg = l.deg;
    a.examined = l.examined;
    const int wpb = 8;
    size_t smem = (size_t)wpb * a.Wr * 4;
    cudaError_t err = cudaSuccess;
    NSG_DISPATCH_DP4(a.dp4, {
        auto kern = prune_entry<G_, V_, U_, PruneBatch<V_>::value>();
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) {
            int per_sm = 0;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
            if (err == cudaSuccess) {
                int64_t need = (l.nv + wpb - 1) / wpb;
                int64_t full = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
                int grid = (int)(need < full ? need : full);
                kern<<<grid, wpb * 32, smem, st>>>(a);
                err = cudaGetLastError();
            }
        }
    });
    return err;
}

// ---------------------------------------------------------------------------
// Reachability from the navigating node: level-synchronous BFS over the
// fixed-width graph (the reached set equals that of the paper's DFS tree).
// ---------------------------------------------------------------------------
__global__ void bfs_seed_kernel(uint32_t *reached, int root, int *frontier, int *count) {
    atomicOr(reached + (root >> 5), 1u << (root & 31));
    frontier[0] = root;
    *count = 1;
}

__global__ void bfs_level_kernel(const int *__restrict__ adj, int R, const int *__restrict__ frontier,
                                 int nf, int *next, int *next_count, uint32_t *reached) {
    const int64_t total = (int64_t)nf * R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int u = frontier[x / R];
        int v = adj[(int64_t)u * R + x % R];
        if (v < 0) continue;
        uint32_t bit = 1u << (v & 31);
        if (!(atomicOr(reached + (v >> 5), bit) & bit)) next[atomicAdd(next_count, 1)] = v;
    }
}

cudaError_t launch_bfs_seed(uint32_t *reached, int root, int *frontier, int *count, cudaStream_t st) {
    bfs_seed_kernel<<<1, 1, 0, st>>>(reached, root, frontier, count);
    return cudaGetLastError();
}

cudaError_t launch_bfs_level(const int *adj, int R, const int *frontier, int nf, int *next,
                             int *next_count, uint32_t *reached, cudaStream_t st) {
    int64_t total = (int64_t)nf * R;
    int64_t blocks = (total + 255) / 256;
    int64_t cap = (int64_t)sm_count() * 8;
    bfs_level_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(adj, R, frontier, nf, next,
                                                                         next_count, reached);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Precision (Eq. 1): per query, how many of the first k ids are among the
// first k ground-truth ids.
// ---------------------------------------------------------------------------
__global__ void recall_kernel(const int *__restrict__ ids, int ld_ids, const int *__restrict__ gt,
                              int ld_gt, int64_t nq, int k, int *hits) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        int h = 0;
        for (int a = 0; a < k; ++a) {
            int id = ids[q * ld_ids + a];
            if (id < 0) continue;
            for (int b = 0; b < k; ++b)
                if (gt[q * ld_gt + b] == id) {
                    ++h;
                    break;
                }
        }
        hits[q] = h;
    }
}

cudaError_t launch_recall(const int *ids, int ld_ids, const int *gt, int ld_gt, int64_t nq, int k,
                          int *hits, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    int64_t blocks = (nq + 255) / 256;
    recall_kernel<<<(int)(blocks < 65535 ? blocks : 65535), 256, 0, st>>>(ids, ld_ids, gt, ld_gt, nq,
                                                                           k, hits);
    return cudaGetLastError();
}

__global__ void pad_rows_kernel(const float *__restrict__ src, int64_t n, int d, float *__restrict__ dst,
                                int dp) {
    const int64_t total = n * dp;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = x / dp;
        int c = (int)(x % dp);
        dst[x] = c < d ? src[r * d + c] : 0.0f;
    }
}

cudaError_t launch_pad_rows(const float *src, int64_t n, int d, float *dst, int dp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n * dp + 255) / 256;
    int64_t cap = (int64_t)sm_count() * 16;
    pad_rows_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(src, n, d, dst, dp);
    return cudaGetLastError();
}

}  // namespace nsg
