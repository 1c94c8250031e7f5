// search_kern.cuh -- the search kernels (Alg. 1 for a batch of queries,
// Section 3.6) and their launch, shared by search.cu (pools in shared
// memory) and search_global.cu (pools in global memory).
#pragma once
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>

#include "kernels.h"
#include "lowp.cuh"
#include "search_core.cuh"
#include "stage.cuh"

// Rows in flight per lane group on the low-precision paths (1 or 2 16-byte
// chunks per lane; NSG_U8ROWS row groups of NSG_U8CHUNKS chunks per lane for
// the 8-bit form).
#ifndef NSG_STOP_MINB
#define NSG_STOP_MINB 3
#endif
#ifndef NSG_UL1
#define NSG_UL1 2
#endif
#ifndef NSG_UL2
#define NSG_UL2 2
#endif
#ifndef NSG_U8ROWS
#define NSG_U8ROWS 3
#endif
#ifndef NSG_U8CHUNKS
#define NSG_U8CHUNKS 2
#endif
#ifndef NSG_U8ROWS_WIDE
#define NSG_U8ROWS_WIDE 8
#endif
#ifndef NSG_UL_WIDE
#define NSG_UL_WIDE 4
#endif
#ifndef NSG_U_RERANK_WIDE
#define NSG_U_RERANK_WIDE 3
#endif

namespace nsg {

__host__ __device__ static inline int round32(int x) { return (x + 31) & ~31; }
static inline int log2i(unsigned x) {
    int r = 0;
    while ((1u << r) < x) ++r;
    return r;
}

struct SearchArgs {
    const float4 *base4;  // FP32 rows [n][dp4] (re-rank and the plain form)
    int dp4;
    const uint4 *lowp;  // BF16 / FP8 / U8 rows [n][dc] 16-byte chunks (precision forms)
    int dc;
    float scale;  // query multiplier matching the low-precision copy
    float lo;     // U8: offset of the 8-bit map
    int rerank;   // precision forms: re-rank the final pool with FP32 rows (1),
                  // U8 only for queries the 8-bit map rounds (2)
    const int *adj;
    int width, W;
    int start;
    const float *queries;
    int d;
    int64_t nq;
    int k, L, H, hshift, max_steps, C;
    int *ids;
    float *d2;
    int *n_expand, *n_dist, *status, *any_capped;
    // learned early termination: FP16 MLP parameters (nullptr: none), logit threshold
    const __half *stop_model;
    float stop_logit;
    int stop_k, stop_min_steps;
    // trace recording: features [nq][cap][NF], change flags [nq][cap]
    float *trace_feat;
    unsigned char *trace_flag;
    int trace_cap;
    // batched uneven queries: per-query k and L (k, L above are the maxima and
    // the output row stride is k), a visiting order and a work counter that
    // persistent warps draw from (nullptr: static grid-stride assignment)
    const int *kv, *Lv, *order;
    int *work;
    // random initial pool (count 0: start at `start`), base rows n
    int init_count;
    uint64_t init_seed;
    int n;
    // partitioned search: unit t searches query t / parts from starts[t % parts]
    int parts;
    const int *starts;
    // global-memory pools: slot (block, warp or group) of L keys, or nullptr
    uint64_t *gpool;
    // staged row gathers (stage.cuh): slots per warp and bytes per slot of
    // each warp's ring, which follows the warps' (groups') regions; a tensor
    // map over the low-precision rows gathers them four per copy (nullptr:
    // one bulk copy per row)
    int stage_nb, stage_rb;
    const CUtensorMap *lmap;
};

// Query row and start node of search unit t.
__device__ __forceinline__ int64_t unit_query(const SearchArgs &a, int64_t t, int *start) {
    if (a.parts > 1) {
        const int64_t q = t / a.parts;
        *start = a.starts[t - q * a.parts];
        return q;
    }
    *start = a.start;
    return t;
}

// The distance functor of precision P for one query (every lane loads its
// share of the query), handed to f.  Returns whether the 8-bit map kept
// every query value (always true for the other forms).
template <bool ST, class D, class F>
__device__ __forceinline__ void run_dist(const D &dist, const StageRef *sr, const CUtensorMap *map, F &&f) {
    if constexpr (ST) {
        const DistStaged<D> sd{dist, *sr, stage_slots(dist, *sr, map != nullptr), dist.row_bytes(), map};
        f(sd);
    } else {
        f(dist);
    }
}

// ST: the rows are gathered through the warp's staging ring *sr (the host
// sizes it for at least one traversal row).
template <int G, int V, int U, int P, bool ST = false, class F>
__device__ __forceinline__ bool with_dist(const SearchArgs &a, const float *qp, const StageRef *sr, F &&f) {
    if constexpr (P == PREC_F32) {
        DistF32<G, V, U> dist{{}, a.base4, a.dp4};
        dist.Q.load(qp, a.d, a.dp4);
        run_dist<ST>(dist, sr, nullptr, f);
        return true;
    } else if constexpr (P == PREC_U8) {
        // an 8-bit row is a quarter of the FP32 row: G8 lanes of up to
        // NSG_U8CHUNKS 16-byte chunks each, 32 / G8 rows per pass
        constexpr int VG = V * G;  // FP32 float4 capacity of a lane group
        constexpr int G8 = VG / (4 * NSG_U8CHUNKS) < 1 ? 1 : (VG / (4 * NSG_U8CHUNKS) > 32 ? 32 : VG / (4 * NSG_U8CHUNKS));
        constexpr int VC = VG / (4 * G8);
        // rows of 513..1024 values run with the default register budget:
        // more of them in flight
        constexpr int U8R = V == 8 ? NSG_U8ROWS_WIDE : (V > 8 ? 2 : NSG_U8ROWS);
        DistU8<G8, VC, U8R> dist{{}, a.lowp, a.dc};
        const bool qexact = dist.Q.load(qp, a.d, a.lo, a.scale);
        run_dist<ST>(dist, sr, a.lmap, f);
        return qexact;
    } else {
        constexpr int VC = (V * 4) / PrecEpc<P>::value > 0 ? (V * 4) / PrecEpc<P>::value : 1;
        // rows in flight per group: a low-precision row costs VC*4 registers per lane
        constexpr int UL = V == 8 ? NSG_UL_WIDE : (VC <= 1 ? NSG_UL1 : (VC == 2 ? NSG_UL2 : 2));
        DistLp<P, G, VC, UL> dist{{}, a.lowp, a.dc};
        dist.Q.load(qp, a.d, a.scale);
        run_dist<ST>(dist, sr, a.lmap, f);
        return true;
    }
}

// After the traversal of query qi (one warp): with `rerank` the L pool
// entries are measured again on the FP32 rows and the k smallest of those
// keys are kept (the re-rank list reuses the visited hash, no longer needed,
// when it has room for k keys, else a list of its own, C = k); then the
// results and counters are written.
// ST: the re-rank gathers its FP32 rows through the staging ring when at
// least one fits there, and a staged copy that never landed (the ring's
// failure word) makes the query's status NSG_ECUDA.
template <int G, int V, int U, int P, bool ST = false>
__device__ __forceinline__ void finish_query(const SearchArgs &a, WarpSmem &s, const SearchOut &o, int64_t qi,
                                             int kq, const float *qp, bool rerank, const StageRef *sr = nullptr) {
    const unsigned lane = lane_id();
    const uint64_t *res = s.pool;
    int rsize = o.size;
    if constexpr (P != PREC_F32) if (rerank) {
        uint64_t *cl = a.C > 0 ? s.clist : reinterpret_cast<uint64_t *>(s.hash);
        // the re-rank gathers all L pool rows at once: more rows in flight
        // than the traversal for rows of 513..1024 values
        // (staged kernels: the ring serves the re-rank; the register gather is
        // only the fallback for a ring too small for one FP32 row)
        constexpr int UR = ST ? 1 : (V == 8 ? NSG_U_RERANK_WIDE : U);
        DistF32<G, V, UR> exact{{}, a.base4, a.dp4};
        exact.Q.load(qp, a.d, a.dp4);
        int kept = 0;
        auto rerank_with = [&](const auto &dist) {
            for (int c0 = 0; c0 < o.size; c0 += a.W) {
                const int mm = o.size - c0 < a.W ? o.size - c0 : a.W;
                for (int t = lane; t < mm; t += 32) s.ids[t] = kid(s.pool[c0 + t]);
                __syncwarp();
                dist(s.ids, mm, s.keys);
                warp_merge(cl, kq, kept, s.keys, mm, s.ck, s.cp, s.sk, s.sp);
            }
        };
        if constexpr (ST) {
            const int nb = stage_slots(exact, *sr);
            if (nb > 0) rerank_with(DistStaged<DistF32<G, V, UR>>{exact, *sr, nb, exact.row_bytes(), nullptr});
            else rerank_with(exact);
        } else {
            rerank_with(exact);
        }
        res = cl;
        rsize = kept;
    }
    for (int c = lane; c < a.k; c += 32) {  // row stride a.k; slots past this query's k padded
        const bool has = c < rsize && c < kq;
        uint64_t e = has ? res[c] : KEY_INF;
        a.ids[qi * a.k + c] = has ? kid(e) : -1;
        if (a.d2) a.d2[qi * a.k + c] = has ? kd2(e) : __int_as_float(0x7f800000);
    }
    if (lane == 0) {
        if (a.n_expand) a.n_expand[qi] = o.n_expand;
        if (a.n_dist) a.n_dist[qi] = o.n_dist;
        bool failed = false;
        if constexpr (ST) failed = sr->state[1] != 0;
        if (a.status) a.status[qi] = failed ? -3 : o.capped ? -4 : 0;
        if (o.capped && a.any_capped) atomicOr(a.any_capped, 1);
    }
    __syncwarp();
}

// Alg. 1 per query, one warp each.  P = PREC_F32: distances on the FP32 rows
// (the plain form).  P = PREC_BF16 / PREC_FP8 / PREC_U8: traversal distances
// on the low-precision copy, then the FP32 re-rank when asked for.
template <int G, int V, int U, int P, bool STOP, bool GP, bool ST = false>
__device__ __forceinline__ void search_body(const SearchArgs &a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    const int Ls = GP ? 0 : a.L;  // pool keys held in shared memory
    const size_t wbytes = warp_smem_bytes(Ls, a.W, a.C, a.H, true);
    WarpSmem s = carve_warp_smem(smem + warp * wbytes, Ls, a.W, a.C, a.H, true);
    if constexpr (GP) s.pool = a.gpool + ((int64_t)blockIdx.x * wpb + warp) * a.L;
    StageRef sref{};
    if constexpr (ST)  // the rings follow the warps' regions (no stop model here)
        sref = stage_init(smem + wpb * wbytes + warp * stage_bytes(a.stage_nb, a.stage_rb), a.stage_nb,
                          a.stage_rb, a.any_capped);
    // the stop model lives after the warps' regions, widened to FP32
    StopMLP *mlp = reinterpret_cast<StopMLP *>(smem + wpb * wbytes);
    if (STOP && a.stop_model != nullptr) {
        float *dst = reinterpret_cast<float *>(mlp);
        for (int t = threadIdx.x; t < NSG_STOP_PARAMS; t += blockDim.x) dst[t] = __half2float(a.stop_model[t]);
        __syncthreads();
    }
    int csize = 0;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    int64_t t = (int64_t)blockIdx.x * wpb + warp;
    for (;;) {
        if (a.work != nullptr) {  // persistent warps draw the next query
            int v = 0;
            if (lane == 0) v = atomicAdd(a.work, 1);
            t = __shfl_sync(NSG_FULL, v, 0);
        }
        if (t >= a.nq) break;
        const int64_t qi = a.order != nullptr ? a.order[t] : t;
        if (a.work == nullptr) t += stride;
        const int kq = a.kv != nullptr ? min(max(a.kv[qi], 1), a.k) : a.k;
        const int Lq = a.Lv != nullptr ? max(min(a.Lv[qi], a.L), kq) : a.L;
        int start;
        const float *qp = a.queries + unit_query(a, qi, &start) * a.d;
        StopCtx sc;
        sc.mlp = a.stop_model != nullptr ? mlp : nullptr;
        sc.logit = a.stop_logit;
        sc.k = a.kv != nullptr ? min(kq, a.stop_k) : a.stop_k;
        sc.min_steps = a.stop_min_steps;
        sc.trace_feat = a.trace_feat != nullptr ? a.trace_feat + qi * (int64_t)a.trace_cap * NSG_STOP_NF : nullptr;
        sc.trace_flag = a.trace_flag != nullptr ? a.trace_flag + qi * (int64_t)a.trace_cap : nullptr;
        sc.trace_cap = a.trace_cap;
        const StopCtx *scp = STOP ? &sc : nullptr;
        const InitRand ir{a.init_count < Lq ? a.init_count : Lq, a.init_seed, qi, a.n};
        const InitRand *initp = a.init_count > 0 ? &ir : nullptr;
        SearchOut o;
        const bool qexact = with_dist<G, V, U, P, ST>(a, qp, &sref, [&](const auto &dist) {
            o = warp_alg1<false, false, std::decay_t<decltype(dist)>, STOP>(
                dist, GraphRef{a.adj, a.width}, start, Lq, s, (uint32_t)a.H - 1, a.hshift, a.max_steps, -1, 0,
                csize, nullptr, 0, scp, nullptr, initp);
        });
        const bool rerank = a.rerank == 1 || (P == PREC_U8 && a.rerank == 2 && !qexact);
        finish_query<G, V, U, P, ST>(a, s, o, qi, kq, qp, rerank, &sref);
    }
}

// Alg. 1 per query by a group of WPQ warps that share the query's pool and
// visited set (group_alg1): WPQ times the rows in flight per expansion, the
// same steps and results.  Group g of a block uses named barrier 1 + g.
struct GroupCtl {
    int64_t t;  // the group's query (drawn by the leader)
    int m, done;
};

template <int G, int V, int U, int P, int WPQ, bool GP, bool ST = false>
__device__ __forceinline__ void search_group_body(const SearchArgs &a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int g = warp / WPQ, w = warp % WPQ, gpb = wpb / WPQ;
    const unsigned lane = lane_id();
    const int Ls = GP ? 0 : a.L;
    const size_t wbytes = warp_smem_bytes(Ls, a.W, a.C, a.H, true);
    WarpSmem s = carve_warp_smem(smem + g * wbytes, Ls, a.W, a.C, a.H, true);
    if constexpr (GP) s.pool = a.gpool + ((int64_t)blockIdx.x * gpb + g) * a.L;
    volatile GroupCtl *ctl = reinterpret_cast<volatile GroupCtl *>(smem + gpb * wbytes) + g;
    StageRef sref{};
    if constexpr (ST) {  // one ring per warp, after the groups' regions and control words
        const size_t off = (gpb * wbytes + gpb * sizeof(GroupCtl) + 15) & ~size_t(15);
        sref = stage_init(smem + off + warp * stage_bytes(a.stage_nb, a.stage_rb), a.stage_nb, a.stage_rb,
                          a.any_capped);
    }
    const int bar_id = 1 + g;
    const int64_t stride = (int64_t)gridDim.x * gpb;
    int64_t tstat = (int64_t)blockIdx.x * gpb + g;
    for (;;) {
        if (w == 0 && lane == 0) ctl->t = a.work != nullptr ? (int64_t)atomicAdd(a.work, 1) : tstat;
        tstat += stride;
        group_bar(bar_id, 32 * WPQ);
        const int64_t t = ctl->t;
        if (t >= a.nq) break;  // the same value in every warp of the group
        const int64_t qi = a.order != nullptr ? a.order[t] : t;
        const int kq = a.kv != nullptr ? min(max(a.kv[qi], 1), a.k) : a.k;
        const int Lq = a.Lv != nullptr ? max(min(a.Lv[qi], a.L), kq) : a.L;
        int start;
        const float *qp = a.queries + unit_query(a, qi, &start) * a.d;
        const InitRand ir{a.init_count < Lq ? a.init_count : Lq, a.init_seed, qi, a.n};
        const InitRand *initp = a.init_count > 0 ? &ir : nullptr;
        SearchOut o;
        const bool qexact = with_dist<G, V, U, P, ST>(a, qp, &sref, [&](const auto &dist) {
            o = group_alg1<WPQ>(dist, GraphRef{a.adj, a.width}, start, Lq, s, (uint32_t)a.H - 1, a.hshift,
                                a.max_steps, w, bar_id, ctl, initp);
        });
        const bool rerank = a.rerank == 1 || (P == PREC_U8 && a.rerank == 2 && !qexact);
        if (w == 0) finish_query<G, V, U, P, ST>(a, s, o, qi, kq, qp, rerank, &sref);
    }
}

// Register budgets.  Rows of up to 512 values (V <= 4 float4 slices per lane)
// are held to 4 blocks of 256 threads per SM, i.e. 64 registers and 32
// resident warps, with no spills; left free, the low-precision kernels (which
// also carry the FP32 re-rank) take ~112 registers and the plain one 70.
// Wider rows (V >= 8) keep the compiler's default budget (~98), since 64 would
// spill.  The learned-stop / trace kernels carry the feature and MLP code and
// are held to 3 blocks per SM (rows up to 512 values) or left free (wider).
template <int G, int V, int U, int P, bool GP>
__global__ void __launch_bounds__(256, 4) search_kernel(SearchArgs a) {
    search_body<G, V, U, P, false, GP>(a);
}
template <int G, int V, int U, int P, bool GP>
__global__ void __launch_bounds__(256) search_wide_kernel(SearchArgs a) {
    search_body<G, V, U, P, false, GP>(a);
}
template <int G, int V, int U, int P, bool GP>
__global__ void __launch_bounds__(256, NSG_STOP_MINB) search_stop_kernel(SearchArgs a) {
    search_body<G, V, U, P, true, GP>(a);
}
template <int G, int V, int U, int P, bool GP>
__global__ void __launch_bounds__(256) search_stop_wide_kernel(SearchArgs a) {
    search_body<G, V, U, P, true, GP>(a);
}
template <int G, int V, int U, int P, int WPQ, bool GP>
__global__ void __launch_bounds__(256, 4) search_group_kernel(SearchArgs a) {
    search_group_body<G, V, U, P, WPQ, GP>(a);
}
template <int G, int V, int U, int P, int WPQ, bool GP>
__global__ void __launch_bounds__(256) search_group_wide_kernel(SearchArgs a) {
    search_group_body<G, V, U, P, WPQ, GP>(a);
}
// Staged row gathers (rows of more than 512 values; stage.cuh).
template <int G, int V, int U, int P, bool GP>
__global__ void __launch_bounds__(256) search_staged_kernel(SearchArgs a) {
    search_body<G, V, U, P, false, GP, true>(a);
}
template <int G, int V, int U, int P, int WPQ, bool GP>
__global__ void __launch_bounds__(256) search_group_staged_kernel(SearchArgs a) {
    search_group_body<G, V, U, P, WPQ, GP, true>(a);
}

// Kernel for precision P at the dispatch shape G, V, U (wpq warps per query;
// the learned-stop / trace kernels run one warp per query), pools in shared
// (GP false) or global memory.
template <int G, int V, int U, int P, bool GP>
static void (*search_entry(bool stop, int wpq))(SearchArgs) {
    if constexpr (V <= 4) {
        if (stop) return search_stop_kernel<G, V, U, P, GP>;
        if (wpq == 2) return search_group_kernel<G, V, U, P, 2, GP>;
        if (wpq == 4) return search_group_kernel<G, V, U, P, 4, GP>;
        return search_kernel<G, V, U, P, GP>;
    } else {
        if (stop) return search_stop_wide_kernel<G, V, U, P, GP>;
        if (wpq == 2) return search_group_wide_kernel<G, V, U, P, 2, GP>;
        if (wpq == 4) return search_group_wide_kernel<G, V, U, P, 4, GP>;
        return search_wide_kernel<G, V, U, P, GP>;
    }
}

template <int G, int V, int U, int P, bool GP>
static void (*staged_entry(int wpq))(SearchArgs) {
    if (wpq == 2) return search_group_staged_kernel<G, V, U, P, 2, GP>;
    if (wpq == 4) return search_group_staged_kernel<G, V, U, P, 4, GP>;
    return search_staged_kernel<G, V, U, P, GP>;
}

template <typename K>
static cudaError_t config(K kernel, size_t smem_per_warp, int want_wpb, int64_t units, int *grid,
                          int *wpb, size_t *smem, size_t smem_per_cta = 0, int step = 1) {
    // warps per block: a multiple of `step` (the warps of one query group)
    size_t cap = smem_optin();
    int w = want_wpb > 0 ? want_wpb : 4;
    w = w < step ? step : w / step * step;
    while (w > step && smem_per_warp * w + smem_per_cta > cap) w -= step;
    if (smem_per_warp * w + smem_per_cta > cap) return cudaErrorInvalidConfiguration;
    *smem = smem_per_warp * w + smem_per_cta;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, w * 32, *smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (units + w - 1) / w;
    int64_t full = (int64_t)sm_count() * per_sm;
    *grid = (int)std::max<int64_t>(1, std::min(need, full));
    *wpb = w;
    return cudaSuccess;
}

// Launch of the search kernels for the launch description `a`: pools in
// shared memory (GP false) or in the global slots a.gpool (GP true, at most
// gpool_slots resident warps or groups); ST: the staged-gather kernels (rows
// of more than 512 values, no stop model).
template <bool GP, bool ST = false>
cudaError_t launch_search_args(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, size_t per_cta,
                               bool stop, int wpq, cudaStream_t st) {
    cudaError_t err = cudaSuccess;
    NSG_DISPATCH_DP4(a.dp4, {
        void (*kern)(SearchArgs) = nullptr;
        if constexpr (ST) {
            if constexpr (V_ >= 8)
                if (!stop)
                    kern = l.precision == PREC_BF16  ? staged_entry<G_, V_, U_, PREC_BF16, GP>(wpq)
                           : l.precision == PREC_FP8 ? staged_entry<G_, V_, U_, PREC_FP8, GP>(wpq)
                           : l.precision == PREC_U8  ? staged_entry<G_, V_, U_, PREC_U8, GP>(wpq)
                                                     : staged_entry<G_, V_, U_, PREC_F32, GP>(wpq);
        } else {
            kern = l.precision == PREC_BF16  ? search_entry<G_, V_, U_, PREC_BF16, GP>(stop, wpq)
                   : l.precision == PREC_FP8 ? search_entry<G_, V_, U_, PREC_FP8, GP>(stop, wpq)
                   : l.precision == PREC_U8  ? search_entry<G_, V_, U_, PREC_U8, GP>(stop, wpq)
                                             : search_entry<G_, V_, U_, PREC_F32, GP>(stop, wpq);
        }
        if (kern == nullptr) return cudaErrorInvalidValue;
        int grid, wpb;
        size_t smem;
        err = config(kern, per_warp, l.warps_per_cta, l.nq * wpq, &grid, &wpb, &smem, per_cta, wpq);
        // a global-memory pool slot per resident warp (group): never more blocks than slots
        if (GP && err == cudaSuccess) {
            const int64_t per_block = wpb / wpq;
            if (l.gpool_slots < per_block) err = cudaErrorInvalidValue;
            else if ((int64_t)grid * per_block > l.gpool_slots) grid = (int)(l.gpool_slots / per_block);
        }
        if (err == cudaSuccess) {
            kern<<<grid, wpb * 32, smem, st>>>(a);
            err = cudaGetLastError();
        }
    });
    return err;
}

// The global-memory and staged instantiations live in translation units of
// their own (search_global.cu, search_staged.cu, search_staged_global.cu) so
// they compile in parallel.
cudaError_t launch_search_global(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, size_t per_cta,
                                 bool stop, int wpq, cudaStream_t st);
cudaError_t launch_search_staged(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, int wpq,
                                 cudaStream_t st);
cudaError_t launch_search_staged_global(const SearchArgs &a, const SearchLaunch &l, size_t per_warp, int wpq,
                                        cudaStream_t st);

}  // namespace nsg
