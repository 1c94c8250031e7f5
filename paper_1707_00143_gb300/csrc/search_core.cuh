// search_core.cuh -- Alg. 1 (Search-on-Graph) for one query per warp.
//
// The pool S is a sorted array of L keys in shared memory (bit 31 of the id =
// checked).  One expansion step: find the first unchecked entry (ballot over
// 32 entries at a time from a cursor before which everything is checked),
// mark it, read its adjacency row, filter the ids through the visited hash,
// compute the distances of the new ids (G-lane groups, U rows in flight per
// group), and merge the new keys into S keeping the L smallest.  The loop
// stops when no unchecked entry is left (reading R1 of the paper's loop
// condition) or when the step cap is reached.
//
// The same routine serves
//   * search on the NSG from the navigating node (Section 3.6),
//   * search-and-collect on the kNN graph (Alg. 2, Section 3.5 iii): every computed
//     key except the node itself is also merged into a collect list of the C
//     smallest keys,
//   * the connectivity pass (Alg. 2, Section 3.5 iv): speculative searches that also
//     log the ids they expand, and re-searches on a graph the same kernel is
//     editing (plain coherent loads instead of the read-only path).
#pragma once

#include "common.cuh"

// L2 prefetch of an expansion's candidate rows before their gather (1 = on):
// the FP32 gather takes several rounds of 8 rows, and the later rounds then
// hit L2.  The 8-bit and BF16 functors gather one or two rounds and skip it.
#ifndef NSG_PF_ROWS
#define NSG_PF_ROWS 1
#endif
// FP32 rows in flight per lane group for rows of 513..1024 values
#ifndef NSG_U_WIDE8
#define NSG_U_WIDE8 2
#endif
// Software pipelining of the expansion loop (searches on a graph nobody edits
// meanwhile): 0 off; 1 the next node's adjacency row is loaded before the
// merge of the current expansion's keys; 2 also filtered through the visited
// set and its new rows prefetched into L2 before the merge.  Off by default:
// at full occupancy the search issues an instruction nearly every cycle, and
// the prediction's extra instructions cost more than the latency they hide
// (SIFT-shaped 1M, 10,000 queries, L = 138: 8-bit form 2.12 ms with 0, 2.39
// with 1, 2.97 with 2; FP32 4.20 / 4.47 / 5.59 ms).
#ifndef NSG_PIPE
#define NSG_PIPE 0
#endif

namespace nsg {

struct WarpSmem {
    uint64_t *pool;   // [L]
    uint64_t *keys;   // [W] keys of the new ids
    uint64_t *ck;     // [W] merge scratch
    uint64_t *sk;     // [W]
    uint64_t *clist;  // [C] collect list (collect mode)
    uint32_t *hash;   // [H]
    int *ids;         // [W] new ids
    int *cp;          // [W]
    int *sp;          // [W]
};

// SHARE_SK: the merge's sorted-key scratch shares the candidate keys' space.
// warp_merge reads its candidates only before it writes sk, so this holds
// wherever one merge consumes the keys -- not in collect mode, where the
// same keys feed the collect list's merge and then the pool's.  The bytes
// saved let the searches hold a larger visited set at full occupancy.
__host__ __device__ inline size_t warp_smem_bytes(int L, int W, int C, int H, bool share_sk = false) {
    size_t b = 8ull * (L + (share_sk ? 2 : 3) * W + C) + 4ull * (H + 3 * W);
    return (b + 15) & ~size_t(15);
}

// Layout per warp: hash first (16-byte aligned for the vector clear; H is a
// power of two >= 4), then the 8-byte arrays, then the int arrays.
__device__ inline WarpSmem carve_warp_smem(unsigned char *p, int L, int W, int C, int H, bool share_sk = false) {
    WarpSmem s;
    s.hash = reinterpret_cast<uint32_t *>(p);
    s.pool = reinterpret_cast<uint64_t *>(s.hash + H);
    s.keys = s.pool + L;
    s.ck = s.keys + W;
    s.sk = share_sk ? s.keys : s.ck + W;
    s.clist = s.ck + (share_sk ? 1 : 2) * W;
    s.ids = reinterpret_cast<int *>(s.clist + C);
    s.cp = s.ids + W;
    s.sp = s.cp + W;
    return s;
}

struct GraphRef {
    const int *adj;  // [n][width], -1 padded
    int width;
};

template <bool COHERENT>
__device__ __forceinline__ int load_adj(const int *p) {
    if (COHERENT) return *reinterpret_cast<const volatile int *>(p);
    return __ldg(p);
}

struct SearchOut {
    int size;      // pool size on exit
    int n_expand;  // nodes checked
    int n_dist;    // distances computed (incl. recomputation after forgetting)
    bool capped;   // step cap reached
    bool stopped;  // the learned stop rule ended the search early
};

// ---------------------------------------------------------------------------
// Learned early termination.  Before each expansion the warp describes the
// search state with NSG_STOP_NF features -- log step count, d(first)/d(k-th),
// d(k-th)/d(next to expand), d(k-th)/d(last), log steps since the first k
// entries last changed, log position of the next entry to expand, new
// neighbours in the last step / width, and whether the last step changed the
// first k -- an MLP (NF -> 64 -> 1, ReLU) maps them to a logit, and the
// search stops when the logit exceeds a threshold.
// With a trace buffer the features and, after the expansion, whether the
// first k_stop pool entries changed are recorded (the training data).
// ---------------------------------------------------------------------------
#define NSG_STOP_NF 8
#ifndef NSG_STOP_EVERY
#define NSG_STOP_EVERY 4
#endif
#define NSG_STOP_H 64
#define NSG_STOP_PARAMS (NSG_STOP_H * NSG_STOP_NF + 2 * NSG_STOP_H + 1)  // w1, b1, w2, b2

struct StopMLP {  // FP32 copy in shared memory
    float w1[NSG_STOP_H][NSG_STOP_NF];
    float b1[NSG_STOP_H];
    float w2[NSG_STOP_H];
    float b2;
};

struct StopCtx {
    const StopMLP *mlp;  // nullptr: no learned stop (trace only)
    float logit;         // stop when the model's logit exceeds this
    int k;               // the result size the rule protects
    int min_steps;
    float *trace_feat;   // [cap][NF] for this query, or nullptr
    unsigned char *trace_flag;  // [cap]
    int trace_cap;
};

__device__ __forceinline__ float stop_logit(const StopMLP &m, const float (&f)[NSG_STOP_NF]) {
    const unsigned lane = lane_id();
    float part = 0.0f;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        float a = m.b1[j];
#pragma unroll
        for (int i = 0; i < NSG_STOP_NF; ++i) a = fmaf(m.w1[j][i], f[i], a);
        part = fmaf(m.w2[j], fmaxf(a, 0.0f), part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(NSG_FULL, part, o);
    return part + m.b2;
}

// Merge keys[0..m) minus id `excl` into the collect list (keys left intact
// for the pool merge that follows).
__device__ __forceinline__ void collect_merge(WarpSmem &s, int m, int excl, int C, int &csize) {
    warp_merge(s.clist, C, csize, s.keys, m, s.ck, s.cp, s.sk, s.sp, excl);
}

// Distances of a query to FP32 rows (the plain form).
template <int G, int V, int U>
struct DistF32 {
    RowQuery<G, V> Q;
    const float4 *base4;
    int dp4;
    __device__ __forceinline__ void operator()(const int *ids, int m, uint64_t *keys) const {
        rows_dist<G, V, U>(Q, base4, dp4, ids, m, keys);
    }
    // rounds of the gather beyond the first exist when m > U * 32 / G
    __device__ __forceinline__ void prefetch(const int *ids, int m) const {
        if (m > U * (32 / G)) prefetch_rows_l2(base4, dp4 * 16, ids, m);
    }
    // every row, ahead of a gather that comes later
    __device__ __forceinline__ void prefetch_all(const int *ids, int m) const {
        prefetch_rows_l2(base4, dp4 * 16, ids, m);
    }
    // Staged gathers (stage.cuh): where row `id` lives, its bytes, and the
    // distance to a copy of it in shared memory -- the lanes' slices and the
    // order of the sums are those of the register gather, so are the keys.
    __device__ __forceinline__ const void *row_addr(int id) const { return base4 + (int64_t)id * dp4; }
    __device__ __forceinline__ int row_bytes() const { return dp4 * 16; }
    __device__ __forceinline__ float row_smem(const unsigned char *row) const {
        const float4 *r = reinterpret_cast<const float4 *>(row);
        const int sub = lane_id() % G;
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int k = t * G + sub;
            s += sq4(k < dp4 ? r[k] : make_float4(0.f, 0.f, 0.f, 0.f), Q.q[t]);
        }
        return group_sum<G>(s);
    }
};

// Seeded random initial pool (NSG-Naive's "Alg. 1 with random
// initialization"): query qi starts from the set of nodes
// splitmix64(seed + qi * 0x9e3779b97f4a7c15 + j) mod n, j < count (count <= L).
struct InitRand {
    int count;
    uint64_t seed;
    int64_t qi;
    int n;
};

// Published SplitMix64 finaliser (Steele, Lea, Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// First unchecked pool entry at or after `cursor` (entries before it are all
// checked), or -1.  Warp-wide.
__device__ __forceinline__ int first_unchecked(const uint64_t *pool, int size, int cursor) {
    const unsigned lane = lane_id();
    for (int b = cursor; b < size; b += 32) {
        const int j = b + (int)lane;
        const bool unchecked = j < size && !(pool[j] & CHK);
        const unsigned bal = __ballot_sync(NSG_FULL, unchecked);
        if (bal) return b + __ffs(bal) - 1;
    }
    return -1;
}

// Reads node u's adjacency row and keeps the neighbours the visited set has
// not seen, in row order, in s.ids; returns their count.  Warp-wide.  The
// first 128 slots are loaded before any visit (the visited-set updates would
// otherwise order each 32-slot load after the previous chunk's), so a row
// costs one global round trip.
template <bool COHERENT>
__device__ __forceinline__ void load_row_head(GraphRef g, int u, int (&vr)[4]) {
    const unsigned lane = lane_id();
    const int *row = g.adj + (int64_t)u * g.width;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int slot = c * 32 + (int)lane;
        vr[c] = slot < g.width ? load_adj<COHERENT>(row + slot) : -1;
    }
}

template <bool COHERENT>
__device__ __forceinline__ int filter_row(GraphRef g, int u, const int (&vr)[4], WarpSmem &s, uint32_t hmask,
                                          int hshift) {
    const unsigned lane = lane_id();
    const int *row = g.adj + (int64_t)u * g.width;
    int m = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c * 32 >= g.width) break;
        const bool fresh = vr[c] >= 0 && visit(s.hash, hmask, hshift, vr[c]);
        const unsigned bal = __ballot_sync(NSG_FULL, fresh);
        if (fresh) s.ids[m + __popc(bal & lanemask_lt())] = vr[c];
        m += __popc(bal);
    }
    for (int b = 128; b < g.width; b += 32) {  // rows wider than 128
        const int slot = b + (int)lane;
        const int v = slot < g.width ? load_adj<COHERENT>(row + slot) : -1;
        const bool fresh = v >= 0 && visit(s.hash, hmask, hshift, v);
        const unsigned bal = __ballot_sync(NSG_FULL, fresh);
        if (fresh) s.ids[m + __popc(bal & lanemask_lt())] = v;
        m += __popc(bal);
    }
    __syncwarp();
    return m;
}

// Reads node u's adjacency row and keeps the neighbours the visited set has
// not seen, in row order, in s.ids; returns their count.  Warp-wide.  The
// first 128 slots are loaded before any visit (the visited-set updates would
// otherwise order each 32-slot load after the previous chunk's), so a row
// costs one global round trip.
template <bool COHERENT>
__device__ __forceinline__ int gather_row(GraphRef g, int u, WarpSmem &s, uint32_t hmask, int hshift) {
    int vr[4];
    load_row_head<COHERENT>(g, u, vr);
    return filter_row<COHERENT>(g, u, vr, s, hmask, hshift);
}

// The node Alg. 1 expands after keys[0..m) are merged into the pool, whose
// entries up to position i are all checked: the smaller of the first
// unchecked entry after i and the smallest new key below the tail of a full
// pool.  ~0 when there is none.  Exact unless that new key equals a pool entry
// (a node the visited set forgot and measured again), which the merge drops:
// the caller checks the prediction against the merged pool.  Warp-wide.
__device__ __forceinline__ uint64_t predict_next(const uint64_t *pool, int size, int L, int i, const uint64_t *keys,
                                                 int m) {
    const unsigned lane = lane_id();
    const uint64_t tail = size >= L ? kval(pool[L - 1]) : ~0ull;
    uint64_t best = ~0ull;
    for (int j = (int)lane; j < m; j += 32) {
        const uint64_t k = keys[j];
        if (k < tail && k < best) best = k;
    }
    const int c = first_unchecked(pool, size, i + 1);
    if (c >= 0 && lane == 0) {
        const uint64_t o = kval(pool[c]);
        if (o < best) best = o;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t x = __shfl_xor_sync(NSG_FULL, best, o);
        best = x < best ? x : best;
    }
    return best;
}

// Takes back the visited-set claims of ids[0..m) (a speculative row filter
// for a node that is not expanded next): the set then has forgotten them,
// which only costs a recomputation, never a skipped node.  Warp-wide.
__device__ __forceinline__ void unvisit_all(WarpSmem &s, uint32_t hmask, int hshift, int m) {
    for (int j = (int)lane_id(); j < m; j += 32) unvisit(s.hash, hmask, hshift, s.ids[j]);
    __syncwarp();
}

// The initial pool: the start node, or the set of `init->count` seeded
// random nodes.  Warp-wide; clears the visited set first.
template <class D>
__device__ __forceinline__ void init_pool(const D &dist, int start, int L, WarpSmem &s, uint32_t hmask, int hshift,
                                          const InitRand *init, SearchOut &o) {
    const unsigned lane = lane_id();
    hash_clear(s.hash, (int)hmask + 1);
    if (init != nullptr && init->count > 0) {
        // the pool starts as the set of the drawn nodes, 32 draws at a time
        for (int b = 0; b < init->count; b += 32) {
            const int j = b + (int)lane;
            const int v = j < init->count
                              ? (int)(splitmix64_dev(init->seed + (uint64_t)init->qi * 0x9e3779b97f4a7c15ull +
                                                     (uint64_t)j) %
                                      (uint64_t)init->n)
                              : -1;
            const bool fresh = v >= 0 && visit(s.hash, hmask, hshift, v);
            const unsigned bal = __ballot_sync(NSG_FULL, fresh);
            if (fresh) s.ids[__popc(bal & lanemask_lt())] = v;
            const int m = __popc(bal);
            __syncwarp();
            if (m > 0) {
                dist(s.ids, m, s.keys);
                o.n_dist += m;
                warp_merge(s.pool, L, o.size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
            }
        }
    } else {
        if (lane == 0) {
            visit(s.hash, hmask, hshift, start);
            s.ids[0] = start;
        }
        __syncwarp();
        dist(s.ids, 1, s.keys);
        o.n_dist = 1;
        if (lane == 0) s.pool[0] = s.keys[0];
        __syncwarp();
        o.size = 1;
    }
}

// Barrier over the first `nthreads` threads that reach named barrier `id`.
__device__ __forceinline__ void group_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Alg. 1 for one query by a group of WPQ warps sharing the pool and visited
// set in shared memory.  Per expansion the leader warp (w == 0) finds the
// node, reads its row and filters it through the visited set; after barrier
// A every warp measures a contiguous slice of the new neighbours; after
// barrier B the leader merges them into the pool.  The steps, keys and merges
// are those of warp_alg1 (one warp), so are the results; the group has WPQ
// times the rows in flight.  Every warp of the group runs the same sequence
// of barriers: the leader's decisions (rows to measure, done) are read from
// `ctl` after barrier A.  The returned counters are the leader's.
template <int WPQ, class D, class Ctl>
__device__ SearchOut group_alg1(const D &dist, GraphRef g, int start, int L, WarpSmem &s, uint32_t hmask,
                                int hshift, int max_steps, int w, int bar_id, volatile Ctl *ctl,
                                const InitRand *init) {
    const unsigned lane = lane_id();
    SearchOut o;
    o.size = 0;
    o.n_expand = 0;
    o.n_dist = 0;
    o.capped = false;
    o.stopped = false;
    if (w == 0) init_pool(dist, start, L, s, hmask, hshift, init, o);
    int cursor = 0, i = -1;
    for (;;) {
        if (w == 0) {
            i = first_unchecked(s.pool, o.size, cursor);
            int m = 0, done = 0;
            if (i < 0) {
                done = 1;
            } else if (o.n_expand >= max_steps) {
                o.capped = true;
                done = 1;
            } else {
                o.n_expand++;
                const uint64_t e = s.pool[i];
                __syncwarp();
                if (lane == 0) s.pool[i] = e | CHK;
                m = gather_row<false>(g, kid(e), s, hmask, hshift);
#if NSG_PF_ROWS
                if (m > 0) dist.prefetch(s.ids, m);
#endif
            }
            if (lane == 0) {
                ctl->m = m;
                ctl->done = done;
            }
            __syncwarp();
        }
        group_bar(bar_id, 32 * WPQ);  // A: the row's new neighbours are in s.ids
        const int m = ctl->m;
        if (ctl->done) break;
        if (m > 0) {
            const int per = (m + WPQ - 1) / WPQ;
            const int lo = w * per;
            const int cnt = m - lo < per ? m - lo : per;
            if (cnt > 0) dist(s.ids + lo, cnt, s.keys + lo);
        }
        group_bar(bar_id, 32 * WPQ);  // B: their keys are in s.keys
        if (w == 0) {
            if (m > 0) {
                o.n_dist += m;
                const int lo = warp_merge(s.pool, L, o.size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
                cursor = min(i + 1, lo);
            } else {
                cursor = i + 1;
            }
        }
    }
    return o;
}

// `dist(ids, m, keys)` writes keys[c] = (d2(query, row ids[c]), ids[c]) for c < m.
// STOP: compile the learned-stop / trace hooks (stop must then be non-null).
//
// Pipelining (NSG_PIPE, graphs nobody edits during the search): once the keys
// of an expansion are known, the node Alg. 1 expands next is predicted
// (predict_next) and its adjacency row is read -- with NSG_PIPE 2 also
// filtered through the visited set, its new rows prefetched into L2 -- before
// the keys are merged into the pool, so those memory round trips overlap the
// merge.  After the merge the first unchecked entry is found as always; when
// it is the predicted node the prepared row is used, otherwise (rare: see
// predict_next) the speculative visited-set claims are taken back and the
// row is read again.  The steps, keys and results are those of the plain loop.
template <bool COLLECT, bool COHERENT, class D, bool STOP = false>
__device__ SearchOut warp_alg1(const D &dist, GraphRef g, int start, int L, WarpSmem &s, uint32_t hmask,
                               int hshift, int max_steps, int excl, int C, int &csize, int *xlog = nullptr,
                               int xcap = 0, const StopCtx *stop = nullptr, uint64_t *xthr = nullptr,
                               const InitRand *init = nullptr) {
    constexpr int PIPE = COHERENT ? 0 : NSG_PIPE;
    const unsigned lane = lane_id();
    SearchOut o;
    o.size = 0;
    o.n_expand = 0;
    o.n_dist = 0;
    o.capped = false;
    o.stopped = false;
    int since_change = 0, last_m = 0;
    bool last_changed = true;
    init_pool(dist, start, L, s, hmask, hshift, init, o);
    if (COLLECT && (init == nullptr || init->count <= 0)) collect_merge(s, 1, excl, C, csize);
    int cursor = 0;
    int pre_u = -1;  // node whose row is prepared (PIPE)
    int pre_m = 0;   // PIPE 2: its new neighbours, already in s.ids
    int vr[4];       // PIPE 1: its first 128 adjacency slots
    for (;;) {
        const int i = first_unchecked(s.pool, o.size, cursor);
        if (i < 0) break;
        if (o.n_expand >= max_steps) {
            o.capped = true;
            break;
        }
        // the learned stop rule is evaluated after stop_min_steps expansions and
        // every NSG_STOP_EVERY after that; traces record features at every one
        if constexpr (STOP) if (stop->trace_feat != nullptr ||
                                (stop->mlp != nullptr && o.n_expand >= stop->min_steps &&
                                 (o.n_expand - stop->min_steps) % NSG_STOP_EVERY == 0)) {
            // state before expanding pool[i]: every lane computes the same features
            const int kk = stop->k < o.size ? stop->k : o.size;
            const float d0 = kd2(s.pool[0]), dk = kd2(s.pool[kk - 1]);
            const float dn = kd2(s.pool[i]), dl = kd2(s.pool[o.size - 1]);
            float f[NSG_STOP_NF];
            f[0] = fminf((float)o.n_expand / (float)L, 4.0f) * 0.25f;  // progress relative to the pool size
            f[1] = dk > 0.0f ? d0 / dk : 1.0f;
            f[2] = dn > 0.0f ? fminf(dk / dn, 4.0f) : 1.0f;
            f[3] = dl > 0.0f ? dk / dl : 1.0f;
            f[4] = log2f(1.0f + (float)since_change) * 0.125f;
            f[5] = (float)i / (float)L;  // position of the next expansion in the pool
            f[6] = (float)last_m / (float)g.width;
            f[7] = last_changed ? 1.0f : 0.0f;
            if (stop->trace_feat != nullptr && o.n_expand < stop->trace_cap) {
                float fv = 0.0f;
#pragma unroll
                for (int t = 0; t < NSG_STOP_NF; ++t)
                    if ((int)lane == t) fv = f[t];
                if (lane < NSG_STOP_NF) stop->trace_feat[(int64_t)o.n_expand * NSG_STOP_NF + lane] = fv;
            }
            if (stop->mlp != nullptr && o.n_expand >= stop->min_steps && stop_logit(*stop->mlp, f) > stop->logit) {
                o.stopped = true;
                break;
            }
        }
        o.n_expand++;
        const uint64_t e = s.pool[i];
        __syncwarp();
        if (lane == 0) s.pool[i] = e | CHK;
        const int u = kid(e);
        if (xlog != nullptr && lane == 0 && o.n_expand <= xcap) {
            xlog[o.n_expand - 1] = u;  // expanded ids
            // and the pool's entry bar at this expansion: a candidate enters
            // only below the L-th key (anything, while the pool is not full)
            if (xthr != nullptr) xthr[o.n_expand - 1] = o.size < L ? KEY_INF : kval(s.pool[L - 1]);
        }
        int m;
        if (PIPE == 2 && u == pre_u) {
            m = pre_m;  // filtered before the previous merge
        } else if (PIPE == 1 && u == pre_u) {
            m = filter_row<COHERENT>(g, u, vr, s, hmask, hshift);
        } else {
            if (PIPE == 2 && pre_u >= 0) unvisit_all(s, hmask, hshift, pre_m);  // mispredicted
            m = gather_row<COHERENT>(g, u, s, hmask, hshift);
        }
        pre_u = -1;
        last_m = m;
#if NSG_PF_ROWS
        if (m > 0 && PIPE != 2) dist.prefetch(s.ids, m);
#endif
        if (m == 0) {
            cursor = i + 1;
            if constexpr (STOP) {  // nothing new: the first k entries are unchanged
                if (stop->trace_flag != nullptr && lane == 0 && o.n_expand <= stop->trace_cap)
                    stop->trace_flag[o.n_expand - 1] = 0;
                last_changed = false;
                ++since_change;
            }
            continue;
        }
        dist(s.ids, m, s.keys);
        o.n_dist += m;
        if (COLLECT) collect_merge(s, m, excl, C, csize);
        if constexpr (PIPE != 0) {
            const uint64_t nx = predict_next(s.pool, o.size, L, i, s.keys, m);
            if (nx != ~0ull && o.n_expand < max_steps) {
                pre_u = kid(nx);
                if constexpr (PIPE == 2) {
                    // s.ids is free: the keys carry their ids
                    __syncwarp();
                    pre_m = gather_row<COHERENT>(g, pre_u, s, hmask, hshift);
                    if (pre_m > 0) dist.prefetch_all(s.ids, pre_m);
                } else {
                    load_row_head<COHERENT>(g, pre_u, vr);
                }
            }
        }
        int lo = warp_merge(s.pool, L, o.size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
        cursor = min(i + 1, lo);
        if constexpr (STOP) {  // did this expansion change the first k entries?
            last_changed = lo < stop->k;
            since_change = last_changed ? 0 : since_change + 1;
            if (stop->trace_flag != nullptr && lane == 0 && o.n_expand <= stop->trace_cap)
                stop->trace_flag[o.n_expand - 1] = last_changed ? 1 : 0;
        }
    }
    // a row prepared for a node that was never expanded (the search ended):
    // its claims leave the visited set, which callers may still consult
    if (PIPE == 2 && pre_u >= 0) unvisit_all(s, hmask, hshift, pre_m);
    __syncwarp();
    return o;
}

// Distance configuration by float4s per row (dp4): group size G, float4
// slices per lane V, rows in flight per group U.
#define NSG_DISPATCH_DP4(dp4, ...)                                              \
    do {                                                                        \
        if ((dp4) <= 8) {                                                       \
            constexpr int G_ = 2, V_ = 4, U_ = 2;                               \
            __VA_ARGS__;                                                        \
        } else if ((dp4) <= 16) {                                               \
            constexpr int G_ = 4, V_ = 4, U_ = 2;                               \
            __VA_ARGS__;                                                        \
        } else if ((dp4) <= 32) {                                               \
            constexpr int G_ = 8, V_ = 4, U_ = 2;                               \
            __VA_ARGS__;                                                        \
        } else if ((dp4) <= 64) {                                               \
            constexpr int G_ = 16, V_ = 4, U_ = 2;                              \
            __VA_ARGS__;                                                        \
        } else if ((dp4) <= 128) {                                              \
            constexpr int G_ = 32, V_ = 4, U_ = 2;                              \
            __VA_ARGS__;                                                        \
        } else if ((dp4) <= 256) {                                              \
            constexpr int G_ = 32, V_ = 8, U_ = NSG_U_WIDE8;                    \
            __VA_ARGS__;                                                        \
        } else {                                                                \
            constexpr int G_ = 32, V_ = 16, U_ = 1;                             \
            __VA_ARGS__;                                                        \
        }                                                                       \
    } while (0)

constexpr int MAX_DP4 = 512;  // d <= 2048

}  // namespace nsg
