// connect.cu -- the connectivity pass of Alg. 2 (Section 3.5 iv).
//
// Sequential definition (what the oracle computes): reach from the
// navigating node; while some node is unreached, u = the smallest unreached
// id, run Alg. 1 on the current graph from the navigating node toward x_u,
// give the first result with a free slot (else the smallest reached id with
// one) the edge s->u, and mark everything u reaches.
//
// GPU form, identical result, in speculate-and-commit batches:
//   gather     the next B unreached ids in ascending order (one CTA);
//   speculate  one warp per listed u runs Alg. 1 on the graph as it stands and
//              keeps its final pool plus the ids it expanded;
//   commit     one CTA walks the list in order: skip u if an earlier fix-up of
//              this batch reached it; reuse its pool unless an edge added since
//              the snapshot could have changed it (then search again on the
//              current graph); pick s from the pool with the current degrees;
//              append s->u; mark what u reaches.
// Alg. 1 reads only the adjacency rows of the nodes it expands, and a new
// edge e->w matters only if e was expanded and w would have entered the pool
// then: the pool was not yet full, or key(w) was below its L-th key at that
// expansion.  Once the pool is full its L-th key never rises, so a w that
// could not enter at e's expansion can never enter later either, and the
// pool is unchanged.  The speculative search logs, per expansion, the node
// and that entry bar; the check uses a relative slack of 2^-10 on the
// distance, so summation-order rounding can only cause an extra re-search.  The list holds consecutive
// unreached ids, so walking it in order and skipping reached ones visits the
// same u sequence as "smallest unreached id" after every fix-up.
#include <climits>
#include <vector>

#include "kernels.h"
#include "search_core.cuh"

// Unreached ids speculated per batch: larger batches run more searches in
// parallel, smaller ones leave fewer earlier fix-ups to make a speculation
// stale.  The batch starts at NSG_CONNECT_BATCH and adapts between
// CONNECT_MIN_BATCH and CONNECT_MAX_BATCH to the share of speculations the
// previous batch had to redo (the result does not depend on it).
#ifndef NSG_CONNECT_U_WIDE8
#define NSG_CONNECT_U_WIDE8 4  // rows in flight per warp, 513..1024-value rows
#endif
#ifndef NSG_CONNECT_BATCH
#define NSG_CONNECT_BATCH 64
#endif

namespace nsg {

namespace {

constexpr int CONNECT_MIN_BATCH = 64;
constexpr int CONNECT_MAX_BATCH = 1024;
constexpr int CONNECT_SQ = 2048;  // queue entries of the reach step held in shared memory

__host__ __device__ inline int round32c(int x) { return (x + 31) & ~31; }
inline int log2c(unsigned x) {
    int r = 0;
    while ((1u << r) < x) ++r;
    return r;
}

template <typename T>
__device__ __forceinline__ T ldv(const T *p) {
    return *reinterpret_cast<const volatile T *>(p);
}

__device__ __forceinline__ bool bit_is_set(const uint32_t *bits, int64_t x) {
    return (ldv(bits + (x >> 5)) >> (x & 31)) & 1u;
}

// ids >= cursor that are not reached, ascending, at most B; meta = {count, last id}
__global__ void __launch_bounds__(256) gather_unreached_kernel(const uint32_t *reached, int64_t n, int64_t cursor,
                                                               int B, int *list, int *meta) {
    __shared__ int warp_sum[8];
    __shared__ int sh_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nwords = (n + 31) >> 5;
    if (tid == 0) sh_total = 0;
    __syncthreads();
    for (int64_t w0 = cursor >> 5; w0 < nwords; w0 += blockDim.x) {
        const int total = sh_total;
        if (total >= B) break;
        const int64_t w = w0 + tid;
        uint32_t miss = 0;
        if (w < nwords) {
            miss = ~ldv(reached + w);
            if (w == nwords - 1 && (n & 31)) miss &= (1u << (n & 31)) - 1u;
            if (w == (cursor >> 5)) miss &= ~((1u << (cursor & 31)) - 1u);
        }
        const int c = __popc(miss);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(NSG_FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        int before = 0, block = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            if (k < warp) before += warp_sum[k];
            block += warp_sum[k];
        }
        int j = total + before + incl - c;
        while (miss && j < B) {
            const int b = __ffs(miss) - 1;
            miss &= miss - 1u;
            list[j++] = (int)(w * 32 + b);
        }
        __syncthreads();
        if (tid == 0) sh_total = total + block;
        __syncthreads();
    }
    if (tid == 0) {
        const int cnt = sh_total < B ? sh_total : B;
        meta[0] = cnt;
        meta[1] = cnt > 0 ? list[cnt - 1] : -1;
    }
}

struct SpecArgs {
    const float4 *base4;
    int dp4;
    const int *adj;
    int R, W, nav, L, H, hshift, max_steps;
    const int *list;
    const int *meta;
    uint64_t *pools;  // [B][L]
    int *psize;       // [B]
    int *xlog;        // [B][xcap]
    uint64_t *xthr;   // [B][xcap]: entry bar of the pool at each expansion
    int *xcnt;        // [B]: expansions, INT_MAX when the search hit its cap
    int xcap;
};

template <int G, int V, int U>
__global__ void __launch_bounds__(256) speculate_kernel(SpecArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    WarpSmem s = carve_warp_smem(smem + warp * warp_smem_bytes(a.L, a.W, 0, a.H), a.L, a.W, 0, a.H);
    const int cnt = a.meta[0];
    int csize = 0;
    for (int j = blockIdx.x * wpb + warp; j < cnt; j += gridDim.x * wpb) {
        const int u = a.list[j];
        DistF32<G, V, U> dist{{}, a.base4, a.dp4};
        dist.Q.load_row(a.base4 + (int64_t)u * a.dp4, a.dp4);
        SearchOut o = warp_alg1<false, false>(dist, GraphRef{a.adj, a.R}, a.nav, a.L, s, (uint32_t)a.H - 1,
                                              a.hshift, a.max_steps, -1, 0, csize, a.xlog + (int64_t)j * a.xcap,
                                              a.xcap, nullptr, a.xthr + (int64_t)j * a.xcap);
        for (int t = lane; t < a.L; t += 32) a.pools[(int64_t)j * a.L + t] = t < o.size ? s.pool[t] : KEY_INF;
        if (lane == 0) {
            a.psize[j] = o.size;
            a.xcnt[j] = o.capped ? INT_MAX : o.n_expand;
        }
        __syncwarp();
    }
}

struct CommitArgs {
    const float4 *base4;
    int dp4;
    int64_t n;
    int *adj, *deg;
    int R, W, nav, L, H, hshift, max_steps;
    uint32_t *reached, *dirty;
    int *deg0;  // out-degree at the start of the batch, valid where dirty
    int *queue;
    const int *list, *meta;
    const uint64_t *pools, *xthr;
    const int *psize, *xlog, *xcnt;
    int xcap;
    int *out;  // [0] edges added, [1] status, [2] capped, [3] re-searched
};

// L1 prefetch of fix-up i's speculative pool and expansion log (written by
// the speculate launch, read-only here), issued one fix-up ahead.
__device__ __forceinline__ void prefetch_fixup(const CommitArgs &a, int i, int xc, int ps) {
    const int pool_lines = (ps * 8 + 127) >> 7, x = xc < a.xcap ? xc : 0;
    const int xlog_lines = (x * 4 + 127) >> 7, xthr_lines = (x * 8 + 127) >> 7;
    for (int t = threadIdx.x; t < pool_lines + xlog_lines + xthr_lines; t += blockDim.x) {
        const char *p = t < pool_lines ? reinterpret_cast<const char *>(a.pools + (int64_t)i * a.L) + (t << 7)
                        : t < pool_lines + xlog_lines
                            ? reinterpret_cast<const char *>(a.xlog + (int64_t)i * a.xcap) + ((t - pool_lines) << 7)
                            : reinterpret_cast<const char *>(a.xthr + (int64_t)i * a.xcap) +
                                  ((t - pool_lines - xlog_lines) << 7);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    }
}

template <int G, int V, int U>
__global__ void __launch_bounds__(256) commit_kernel(CommitArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sh_flag, sh_found, sh_size, sh_qtail;
    __shared__ int s_list[CONNECT_MAX_BATCH], s_xcnt[CONNECT_MAX_BATCH], s_psize[CONNECT_MAX_BATCH];
    __shared__ int sq[CONNECT_SQ];  // the reach step's queue (entries past it in a.queue)
    const int tid = threadIdx.x, warp = tid >> 5;
    WarpSmem s = carve_warp_smem(smem, a.L, a.W, 0, a.H);
    const int cnt = a.meta[0];
    for (int t = tid; t < cnt; t += blockDim.x) {
        s_list[t] = a.list[t];
        s_xcnt[t] = a.xcnt[t];
        s_psize[t] = a.psize[t];
    }
    __syncthreads();
    if (cnt > 0) prefetch_fixup(a, 0, s_xcnt[0], s_psize[0]);
    int added = 0, redone = 0, status = 0, capped = 0;
    for (int i = 0; i < cnt; ++i) {
        const int u = s_list[i];
        if (i + 1 < cnt) prefetch_fixup(a, i + 1, s_xcnt[i + 1], s_psize[i + 1]);
        if (bit_is_set(a.reached, u)) continue;  // reached by an earlier fix-up of this batch
        if (tid == 0) sh_flag = 0;
        __syncthreads();
        const int xc = s_xcnt[i];
        if (xc > a.xcap) {
            if (tid == 0) sh_flag = 1;
        } else {
            const float4 *xu = a.base4 + (int64_t)u * a.dp4;
            for (int t = tid; t < xc; t += blockDim.x) {
                const int e = a.xlog[(int64_t)i * a.xcap + t];
                if (!bit_is_set(a.dirty, e)) continue;
                const uint64_t thr = a.xthr[(int64_t)i * a.xcap + t];
                if (thr == KEY_INF) {  // the pool was not full: any new neighbour entered
                    sh_flag = 1;
                    continue;
                }
                const float bar = kd2(thr) * (1.0f + 1.0f / 1024.0f);
                const int d1 = ldv(a.deg + e);
                for (int j = ldv(a.deg0 + e); j < d1; ++j) {
                    const int w = ldv(a.adj + (int64_t)e * a.R + j);
                    const float4 *xw = a.base4 + (int64_t)w * a.dp4;
                    float d2 = 0.0f;
                    for (int c = 0; c < a.dp4; ++c) {
                        const float4 p = xu[c], q = xw[c];
                        const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z, dw = p.w - q.w;
                        d2 += dx * dx + dy * dy + dz * dz + dw * dw;
                    }
                    if (d2 <= bar) sh_flag = 1;
                }
            }
        }
        __syncthreads();
        const uint64_t *pool;
        int size;
        if (sh_flag) {  // the snapshot is stale for this u: search the current graph
            if (warp == 0) {
                DistF32<G, V, U> dist{{}, a.base4, a.dp4};
                dist.Q.load_row(a.base4 + (int64_t)u * a.dp4, a.dp4);
                int csize = 0;
                SearchOut o = warp_alg1<false, true>(dist, GraphRef{a.adj, a.R}, a.nav, a.L, s, (uint32_t)a.H - 1,
                                                     a.hshift, a.max_steps, -1, 0, csize);
                if (lane_id() == 0) {
                    sh_size = o.size;
                    if (o.capped) sh_flag = 2;
                }
            }
            __syncthreads();
            pool = s.pool;
            size = sh_size;
            ++redone;
            if (sh_flag == 2) capped = 1;
        } else {
            pool = a.pools + (int64_t)i * a.L;
            size = s_psize[i];
        }
        // first pool entry (key order) whose out-degree is below R
        if (tid == 0) sh_found = INT_MAX;
        __syncthreads();
        for (int t = tid; t < size; t += blockDim.x)
            if (ldv(a.deg + kid(pool[t])) < a.R) atomicMin(&sh_found, t);
        __syncthreads();
        int sel = sh_found == INT_MAX ? -1 : kid(pool[sh_found]);
        __syncthreads();
        if (sel < 0) {  // else the smallest reached id with a free slot
            if (tid == 0) sh_found = INT_MAX;
            __syncthreads();
            for (int64_t x = tid; x < a.n; x += blockDim.x)
                if (bit_is_set(a.reached, x) && ldv(a.deg + x) < a.R) atomicMin(&sh_found, (int)x);
            __syncthreads();
            sel = sh_found == INT_MAX ? -1 : sh_found;
            __syncthreads();
            if (sel < 0) {
                status = -5;
                break;
            }
        }
        if (tid == 0) {
            const int dg = a.deg[sel];
            a.adj[(int64_t)sel * a.R + dg] = u;
            a.deg[sel] = dg + 1;
            if (!(atomicOr(a.dirty + (sel >> 5), 1u << (sel & 31)) & (1u << (sel & 31)))) a.deg0[sel] = dg;
            atomicOr(a.reached + (u >> 5), 1u << (u & 31));
            sq[0] = u;
            sh_qtail = 1;
        }
        ++added;
        __syncthreads();
        int head = 0;  // mark everything u reaches
        for (;;) {
            const int tail = sh_qtail;
            if (head == tail) break;
            __syncthreads();
            const int64_t total = (int64_t)(tail - head) * a.R;
            for (int64_t x = tid; x < total; x += blockDim.x) {
                const int qi = head + (int)(x / a.R);
                const int node = qi < CONNECT_SQ ? sq[qi] : ldv(a.queue + qi);
                const int v = ldv(a.adj + (int64_t)node * a.R + x % a.R);
                if (v < 0) continue;
                const uint32_t bit = 1u << (v & 31);
                if (!(atomicOr(a.reached + (v >> 5), bit) & bit)) {
                    const int at = atomicAdd(&sh_qtail, 1);
                    if (at < CONNECT_SQ) sq[at] = v;
                    else a.queue[at] = v;
                }
            }
            head = tail;
            __syncthreads();
        }
    }
    if (tid == 0) {
        a.out[0] += added;
        if (status) a.out[1] = status;
        a.out[2] |= capped;
        a.out[3] += redone;
    }
}

template <typename T>
struct Buf {
    T *p = nullptr;
    ~Buf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T)); }
};

}  // namespace

cudaError_t run_connect(const ConnectLaunch &l, int out_host[4], cudaStream_t st) {
    const int64_t n = l.n;
    const int64_t nwords = (n + 31) / 32;
    const int BMAX = CONNECT_MAX_BATCH;
    int B = NSG_CONNECT_BATCH < CONNECT_MIN_BATCH ? CONNECT_MIN_BATCH
            : NSG_CONNECT_BATCH > BMAX            ? BMAX
                                                  : NSG_CONNECT_BATCH;
    const int xcap = 4 * l.L + 64;
    Buf<uint32_t> reached, dirty;
    Buf<int> qa, qb, cnt, list, meta, psize, xlog, xcnt, out, deg0;
    Buf<uint64_t> pools, xthr;
    cudaError_t e;
    if ((e = reached.alloc(nwords)) || (e = dirty.alloc(nwords)) || (e = qa.alloc(n)) || (e = qb.alloc(n)) ||
        (e = cnt.alloc(2)) || (e = list.alloc(BMAX)) || (e = meta.alloc(2)) || (e = psize.alloc(BMAX)) ||
        (e = xlog.alloc((size_t)BMAX * xcap)) || (e = xcnt.alloc(BMAX)) || (e = out.alloc(4)) ||
        (e = pools.alloc((size_t)BMAX * l.L)) || (e = xthr.alloc((size_t)BMAX * xcap)) || (e = deg0.alloc(n)))
        return e;
    if ((e = cudaMemsetAsync(reached.p, 0, nwords * 4, st)) || (e = cudaMemsetAsync(out.p, 0, 16, st))) return e;
    // reach from the navigating node: level-synchronous BFS
    if ((e = launch_bfs_seed(reached.p, l.nav, qa.p, cnt.p, st))) return e;
    int nf = 1;
    int *cur = qa.p, *nxt = qb.p;
    for (int64_t level = 0; nf > 0 && level <= n; ++level) {
        if ((e = cudaMemsetAsync(cnt.p + 1, 0, sizeof(int), st))) return e;
        if ((e = launch_bfs_level(l.adj, l.R, cur, nf, nxt, cnt.p + 1, reached.p, st))) return e;
        if ((e = cudaMemcpyAsync(&nf, cnt.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        std::swap(cur, nxt);
    }
    SpecArgs sa;
    sa.base4 = reinterpret_cast<const float4 *>(l.base);
    sa.dp4 = l.dp / 4;
    sa.adj = l.adj;
    sa.R = l.R;
    sa.W = round32c(l.R);
    sa.nav = l.nav;
    sa.L = l.L;
    sa.H = l.hash_slots;
    sa.hshift = 32 - log2c((unsigned)l.hash_slots);
    sa.max_steps = l.max_steps;
    sa.list = list.p;
    sa.meta = meta.p;
    sa.pools = pools.p;
    sa.psize = psize.p;
    sa.xlog = xlog.p;
    sa.xthr = xthr.p;
    sa.xcnt = xcnt.p;
    sa.xcap = xcap;
    CommitArgs ca;
    ca.base4 = sa.base4;
    ca.dp4 = sa.dp4;
    ca.n = n;
    ca.adj = l.adj;
    ca.deg = l.deg;
    ca.R = l.R;
    ca.W = sa.W;
    ca.nav = l.nav;
    ca.L = l.L;
    ca.H = sa.H;
    ca.hshift = sa.hshift;
    ca.max_steps = l.max_steps;
    ca.reached = reached.p;
    ca.dirty = dirty.p;
    ca.deg0 = deg0.p;
    ca.queue = qa.p;
    ca.list = list.p;
    ca.meta = meta.p;
    ca.pools = pools.p;
    ca.psize = psize.p;
    ca.xlog = xlog.p;
    ca.xthr = xthr.p;
    ca.xcnt = xcnt.p;
    ca.xcap = xcap;
    ca.out = out.p;
    const size_t per_warp = warp_smem_bytes(l.L, sa.W, 0, sa.H);
    const int wpb = 4;
    int64_t cursor = 0;
    int prev[4] = {0, 0, 0, 0};
    for (int64_t batch = 0; batch <= n; ++batch) {
        gather_unreached_kernel<<<1, 256, 0, st>>>(reached.p, n, cursor, B, list.p, meta.p);
        if ((e = cudaGetLastError())) return e;
        int h[2] = {0, 0};
        if ((e = cudaMemcpyAsync(h, meta.p, sizeof(h), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        if (h[0] == 0) break;
        cursor = (int64_t)h[1] + 1;
        if ((e = cudaMemsetAsync(dirty.p, 0, nwords * 4, st))) return e;
        NSG_DISPATCH_DP4(sa.dp4, {
            // one batch runs only 64 searches, so their latency, not the
            // occupancy, sets the time: 513..1024-value rows keep more rows
            // in flight than the search kernels do
            constexpr int UC = V_ == 8 ? NSG_CONNECT_U_WIDE8 : U_;
            auto spec = speculate_kernel<G_, V_, UC>;
            auto commit = commit_kernel<G_, V_, UC>;
            if (!e) e = cudaFuncSetAttribute(spec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per_warp * wpb));
            if (!e) e = cudaFuncSetAttribute(commit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)per_warp);
            if (!e) {
                const int grid = (h[0] + wpb - 1) / wpb;
                spec<<<grid, wpb * 32, per_warp * wpb, st>>>(sa);
                commit<<<1, 256, per_warp, st>>>(ca);
                e = cudaGetLastError();
            }
        });
        if (e) return e;
        int o[4];
        if ((e = cudaMemcpyAsync(o, out.p, sizeof(o), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        if (o[1]) break;
        // a speculation redone in the commit costs a whole serial search, a
        // larger batch saves a share of one parallel search per fix-up: grow the
        // batch while at most 1 in 100 speculations were redone, in this batch
        // and overall, shrink it when more than 1 in 50 of this batch's were
        // (SIFT-shaped 1M: ~1.8 % at 64, which stays; DEEP-shaped 10M and
        // GAUSS5M: < 0.5 % up to 1,024, connectivity 16.4 -> 8.4 s and
        // 19.2 -> 5.3 s)
        const int fixed = o[0] - prev[0], redone = o[3] - prev[3];
        if (redone * 100 <= fixed && o[3] * 100 <= o[0] && B < BMAX) B *= 2;
        else if (redone * 50 > fixed && B > CONNECT_MIN_BATCH) B /= 2;
        for (int t = 0; t < 4; ++t) prev[t] = o[t];
    }
    if ((e = cudaMemcpyAsync(out_host, out.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace nsg
