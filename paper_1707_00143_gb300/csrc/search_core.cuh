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
//   * search on the NSG from the navigating node (Section 3.5),
//   * search-and-collect on the kNN graph (Alg. 2 lines 5-6): every computed
//     key except the node itself is also merged into a collect list of the C
//     smallest keys,
//   * the connectivity pass (Alg. 2 line 26): speculative searches that also
//     log the ids they expand, and re-searches on a graph the same kernel is
//     editing (plain coherent loads instead of the read-only path).
#pragma once

#include "common.cuh"

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

__host__ __device__ inline size_t warp_smem_bytes(int L, int W, int C, int H) {
    size_t b = 8ull * (L + 3 * W + C) + 4ull * (H + 3 * W);
    return (b + 15) & ~size_t(15);
}

// Layout per warp: hash first (16-byte aligned for the vector clear; H is a
// power of two >= 4), then the 8-byte arrays, then the int arrays.
__device__ inline WarpSmem carve_warp_smem(unsigned char *p, int L, int W, int C, int H) {
    WarpSmem s;
    s.hash = reinterpret_cast<uint32_t *>(p);
    s.pool = reinterpret_cast<uint64_t *>(s.hash + H);
    s.keys = s.pool + L;
    s.ck = s.keys + W;
    s.sk = s.ck + W;
    s.clist = s.sk + W;
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
};

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
};

// `dist(ids, m, keys)` writes keys[c] = (d2(query, row ids[c]), ids[c]) for c < m.
template <bool COLLECT, bool COHERENT, class D>
__device__ SearchOut warp_alg1(const D &dist, GraphRef g, int start, int L, WarpSmem &s, uint32_t hmask,
                               int hshift, int max_steps, int excl, int C, int &csize, int *xlog = nullptr,
                               int xcap = 0) {
    const unsigned lane = lane_id();
    SearchOut o;
    o.size = 0;
    o.n_expand = 0;
    o.n_dist = 0;
    o.capped = false;
    hash_clear(s.hash, (int)hmask + 1);
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
    if (COLLECT) collect_merge(s, 1, excl, C, csize);
    int cursor = 0;
    for (;;) {
        int i = -1;
        for (int b = cursor; b < o.size; b += 32) {
            int j = b + (int)lane;
            bool unchecked = j < o.size && !(s.pool[j] & CHK);
            unsigned bal = __ballot_sync(NSG_FULL, unchecked);
            if (bal) {
                i = b + __ffs(bal) - 1;
                break;
            }
        }
        if (i < 0) break;
        if (o.n_expand >= max_steps) {
            o.capped = true;
            break;
        }
        o.n_expand++;
        const uint64_t e = s.pool[i];
        __syncwarp();
        if (lane == 0) s.pool[i] = e | CHK;
        const int u = kid(e);
        if (xlog != nullptr && lane == 0 && o.n_expand <= xcap) xlog[o.n_expand - 1] = u;  // expanded ids
        const int *row = g.adj + (int64_t)u * g.width;
        int m = 0;
        for (int b = 0; b < g.width; b += 32) {
            int slot = b + (int)lane;
            int v = slot < g.width ? load_adj<COHERENT>(row + slot) : -1;
            bool fresh = v >= 0 && visit(s.hash, hmask, hshift, v);
            unsigned bal = __ballot_sync(NSG_FULL, fresh);
            if (fresh) s.ids[m + __popc(bal & lanemask_lt())] = v;
            m += __popc(bal);
        }
        __syncwarp();
        if (m == 0) {
            cursor = i + 1;
            continue;
        }
        dist(s.ids, m, s.keys);
        o.n_dist += m;
        if (COLLECT) collect_merge(s, m, excl, C, csize);
        int lo = warp_merge(s.pool, L, o.size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
        cursor = min(i + 1, lo);
    }
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
            constexpr int G_ = 32, V_ = 8, U_ = 2;                              \
            __VA_ARGS__;                                                        \
        } else {                                                                \
            constexpr int G_ = 32, V_ = 16, U_ = 1;                             \
            __VA_ARGS__;                                                        \
        }                                                                       \
    } while (0)

constexpr int MAX_DP4 = 512;  // d <= 2048

}  // namespace nsg
