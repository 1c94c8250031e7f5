// common.cuh -- device building blocks shared by the NSG kernels (sm_103a).
//
// Keys.  A candidate is the 64-bit key (float bits of d2) << 32 | id.  Squared
// distances are >= +0, so the unsigned order of the key is exactly the
// (distance, id) order the method sorts by (Alg. 1; lower index on ties as in
// the MRNG definition).  Bit 31 of the id word marks "checked" inside a search
// pool and is masked out of every comparison.
#pragma once

#include <climits>

#include <cuda_runtime.h>
#include <stdint.h>

#define NSG_FULL 0xffffffffu

namespace nsg {

constexpr uint64_t CHK = 0x80000000ull;
constexpr uint64_t KEY_INF = 0x7f800000ffffffffull;  // +inf, id -1 (sorts last among finite)
constexpr uint32_t HASH_EMPTY = 0xffffffffu;

__device__ __forceinline__ uint64_t make_key(float d2, int id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint32_t)id;
}
__device__ __forceinline__ uint64_t kval(uint64_t k) { return k & ~CHK; }
__device__ __forceinline__ int kid(uint64_t k) { return (int)(uint32_t)(k & 0x7fffffffull); }
__device__ __forceinline__ float kd2(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// Row distances.  A warp is split into groups of G lanes; each group owns one
// row at a time and each lane holds V float4 slices of the query (slice t of
// lane `sub` covers float4 index t*G + sub, so one load instruction of a group
// reads G consecutive 16-byte chunks).  dp4 = float4s per row.
// ---------------------------------------------------------------------------
template <int G, int V>
struct RowQuery {
    float4 q[V];

    // Load a query of d floats (any d, any 4-byte alignment), zero padded.
    __device__ __forceinline__ void load(const float *__restrict__ src, int d, int dp4) {
        const int sub = lane_id() % G;
#pragma unroll
        for (int t = 0; t < V; ++t) {
            int c = t * G + sub;
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int j = c * 4 + e;
                v[e] = (c < dp4 && j < d) ? __ldg(src + j) : 0.0f;
            }
            q[t] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }

    // Load a padded base row (dp4 float4s, 16-byte aligned).
    __device__ __forceinline__ void load_row(const float4 *__restrict__ row, int dp4) {
        const int sub = lane_id() % G;
#pragma unroll
        for (int t = 0; t < V; ++t) {
            int c = t * G + sub;
            q[t] = (c < dp4) ? __ldg(row + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
};

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(NSG_FULL, v, o, G);
    return v;
}

__device__ __forceinline__ float sq4(float4 a, float4 b) {
    float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z, w = a.w - b.w;
    return x * x + y * y + z * z + w * w;
}

// Squared distances from the query to rows ids[0..m) (smem list); keys[c] is
// written for each c.  U rows per group are in flight at once.
template <int G, int V, int U>
__device__ __forceinline__ void rows_dist(const RowQuery<G, V> &Q, const float4 *__restrict__ base4,
                                          int dp4, const int *ids, int m, uint64_t *keys) {
    constexpr int P = 32 / G;
    const int lane = lane_id(), grp = lane / G, sub = lane % G;
    for (int c0 = 0; c0 < m; c0 += P * U) {
        float4 x[U][V];
        int id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int c = c0 + u * P + grp;
            id[u] = c < m ? ids[c] : -1;
            const float4 *row = base4 + (int64_t)(id[u] < 0 ? 0 : id[u]) * dp4;
#pragma unroll
            for (int t = 0; t < V; ++t) {
                int k = t * G + sub;
                x[u][t] = (id[u] >= 0 && k < dp4) ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float s = 0.0f;
#pragma unroll
            for (int t = 0; t < V; ++t) s += sq4(x[u][t], Q.q[t]);
            s = group_sum<G>(s);
            int c = c0 + u * P + grp;
            if (sub == 0 && c < m) keys[c] = make_key(s, id[u]);
        }
    }
    __syncwarp();
}

// L2 prefetch of the 128-byte lines of rows ids[0..m) (row_bytes each): the
// lanes split the (row, line) pairs.  Issued before a gather that takes
// several rounds, it lets the later rounds hit L2 instead of HBM.
__device__ __forceinline__ void prefetch_rows_l2(const void *base, int row_bytes, const int *ids, int m) {
    const int lines = (row_bytes + 127) >> 7;
    const int total = m * lines;
    for (int x = lane_id(); x < total; x += 32) {
        const int r = x / lines, l = x - r * lines;
        const char *p = static_cast<const char *>(base) + (int64_t)ids[r] * row_bytes + (l << 7);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

// ---------------------------------------------------------------------------
// Visited set of full 32-bit ids, so it never reports a node it has not seen.
// It may forget one: a forgotten node has its distance computed again, which
// yields the identical key (dropped as a duplicate by warp_merge, or rejected
// by the pool tail), so results do not change -- only the distance count grows.
//
// NSG_HASH_WAYS = 4 (default): slots/4 buckets of 4 ids (one 16-byte word),
// probed in order from the home bucket, at most HASH_BUCKET_PROBES buckets
// (default 1: measured fastest, the recomputations cost less than the probes);
// a lookup is one 16-byte shared load per bucket.  An id is claimed into the
// first empty slot of the first bucket that has one (compare-and-swap, so
// lanes of one warp inserting into one bucket at once all keep their ids);
// when every probed bucket is full it is shifted into the home bucket (the
// bucket's oldest id is forgotten).  A bucket never becomes non-full again,
// so a lookup may stop at the first bucket with an empty slot.  Two lanes
// offering one id at once (a row listing it twice): the compare-and-swap
// gives it to one of them; on the overwrite path both may report it new, and
// warp_merge drops the second copy.
// NSG_HASH_WAYS = 0: linear probing over single slots with compare-and-swap,
// 8 probes, then the home slot is overwritten.
// ---------------------------------------------------------------------------
#ifndef NSG_HASH_WAYS
#define NSG_HASH_WAYS 4
#endif
constexpr int HASH_PROBES = 8;
#ifndef NSG_HASH_BUCKET_PROBES
#define NSG_HASH_BUCKET_PROBES 1
#endif
constexpr int HASH_BUCKET_PROBES = NSG_HASH_BUCKET_PROBES;

__device__ __forceinline__ uint4 lds_volatile_u4(const uint4 *p) {
    uint4 v;
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

__device__ __forceinline__ bool visit(uint32_t *h, uint32_t mask, int shift, int id) {
    const uint32_t u = (uint32_t)id;
#if NSG_HASH_WAYS == 4
    const uint32_t bmask = mask >> 2;  // buckets - 1
    const uint32_t home = (u * 2654435761u) >> (shift + 2);
    uint4 *b4 = reinterpret_cast<uint4 *>(h);
    uint32_t b = home;
    uint4 e0 = make_uint4(0, 0, 0, 0);
#pragma unroll 1
    for (int t = 0; t < HASH_BUCKET_PROBES; ++t) {
#pragma unroll 1
        for (int tries = 0; tries < 4; ++tries) {  // each failed claim fills one more slot
            const uint4 e = lds_volatile_u4(b4 + b);
            if (t == 0) e0 = e;
            if (e.x == u || e.y == u || e.z == u || e.w == u) return false;
            const int j = e.x == HASH_EMPTY ? 0 : e.y == HASH_EMPTY ? 1 : e.z == HASH_EMPTY ? 2 : e.w == HASH_EMPTY ? 3 : -1;
            if (j < 0) break;  // full: next bucket
            const uint32_t old = atomicCAS(h + b * 4 + j, HASH_EMPTY, u);
            if (old == HASH_EMPTY) return true;
            if (old == u) return false;
        }
        b = (b + 1) & bmask;
    }
    b4[home] = make_uint4(u, e0.x, e0.y, e0.z);
    return true;
#else
    uint32_t home = (u * 2654435761u) >> shift;
    uint32_t s = home;
#pragma unroll 1
    for (int t = 0; t < HASH_PROBES; ++t) {
        uint32_t old = atomicCAS(&h[s], HASH_EMPTY, u);
        if (old == HASH_EMPTY) return true;
        if (old == u) return false;
        s = (s + 1) & mask;
    }
    atomicExch(&h[home], u);
    return true;
#endif
}

// Removes id from the visited set if it is there (the set forgets it: a later
// visit reports it new, so its distance is measured again).  Not concurrent
// with visit() by other lanes on the same id.
__device__ __forceinline__ void unvisit(uint32_t *h, uint32_t mask, int shift, int id) {
    const uint32_t u = (uint32_t)id;
#if NSG_HASH_WAYS == 4
    const uint32_t bmask = mask >> 2;
    uint32_t b = (u * 2654435761u) >> (shift + 2);
#pragma unroll 1
    for (int t = 0; t < HASH_BUCKET_PROBES; ++t) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (h[b * 4 + j] == u) h[b * 4 + j] = HASH_EMPTY;
        b = (b + 1) & bmask;
    }
#else
    uint32_t s = (u * 2654435761u) >> shift;
#pragma unroll 1
    for (int t = 0; t < HASH_PROBES; ++t) {
        if (h[s] == u) h[s] = HASH_EMPTY;
        s = (s + 1) & mask;
    }
#endif
}

__device__ __forceinline__ void hash_clear(uint32_t *h, int slots) {
    uint4 *h4 = reinterpret_cast<uint4 *>(h);
    const uint4 e = make_uint4(HASH_EMPTY, HASH_EMPTY, HASH_EMPTY, HASH_EMPTY);
    for (int i = lane_id(); i < slots / 4; i += 32) h4[i] = e;
    __syncwarp();
}

// ---------------------------------------------------------------------------
// warp_merge: merge m candidate keys cand[0..m) into the sorted list
// list[0..size) of capacity cap ("add, sort ascending, keep the first cap").
// Candidates not below the tail of a full list, candidates equal to a list
// entry (checked flag ignored) or to an earlier candidate, and id `excl` are
// dropped.  Scratch ck/sk (u64) and cp/sp (int) need m entries each.  Returns
// the smallest position written (cap when nothing entered).  All 32 lanes
// must call it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_key(const uint64_t *list, int size, uint64_t k) {
    int lo = 0, hi = size;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (kval(list[mid]) < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int count_le(const int *sp, int m, int i) {
    int lo = 0, hi = m;  // number of r with sp[r] <= i (sp non-decreasing)
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sp[mid] <= i) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int warp_merge(uint64_t *list, int cap, int &size, const uint64_t *cand,
                                          int m, uint64_t *ck, int *cp, uint64_t *sk, int *sp,
                                          int excl = -1) {
    const unsigned lane = lane_id();
    const uint64_t tail = (size >= cap) ? kval(list[cap - 1]) : ~0ull;
    int nk = 0;
    for (int b = 0; b < m; b += 32) {
        int j = b + lane;
        bool keep = false;
        uint64_t k = 0;
        int p = 0;
        if (j < m) {
            k = cand[j];
            keep = k < tail && kid(k) != excl;
            if (keep) {
                p = lower_bound_key(list, size, k);
                if (p < size && kval(list[p]) == k) keep = false;
            }
        }
        unsigned bal = __ballot_sync(NSG_FULL, keep);
        if (keep) {
            int o = nk + __popc(bal & lanemask_lt());
            ck[o] = k;
            cp[o] = p;
        }
        nk += __popc(bal);
    }
    __syncwarp();
    if (nk == 0) return cap;
    // rank among the kept candidates (stable on equal keys): the number of
    // smaller keys plus the number of equal keys before it
    bool dup = false;
    if (nk <= 32) {
        // one candidate per lane; equal keys (the same node offered twice)
        // found with one match instruction instead of a second compare per key
        const uint64_t k = (int)lane < nk ? ck[lane] : ~0ull;  // ~0: no key
        int r = 0;
#pragma unroll 4
        for (int i = 0; i < nk; ++i) r += ck[i] < k;
        const int before = __popc(__match_any_sync(NSG_FULL, k) & lanemask_lt());
        if ((int)lane < nk) {
            r += before;
            dup = before > 0;
            sk[r] = k;
            sp[r] = cp[lane];
        }
    } else {
        for (int j = lane; j < nk; j += 32) {
            uint64_t k = ck[j];
            int r = 0;
            for (int i = 0; i < nk; ++i) {
                uint64_t o = ck[i];
                const bool same_before = o == k && i < j;
                r += (o < k) || same_before;
                dup |= same_before;
            }
            sk[r] = k;
            sp[r] = cp[j];
        }
    }
    __syncwarp();
    if (__any_sync(NSG_FULL, dup)) {
        // one node offered twice in this batch (a row that lists an id twice):
        // equal keys sit next to each other in sk; keep the first of each run
        int w = 0;
        uint64_t before = ~0ull;  // original key just below this chunk
        for (int b = 0; b < nk; b += 32) {
            const int j = b + (int)lane;
            uint64_t k = 0;
            int p = 0;
            bool keep = false;
            if (j < nk) {
                k = sk[j];
                p = sp[j];
                const uint64_t prev = lane == 0 ? before : sk[j - 1];
                keep = j == 0 || prev != k;
            }
            before = __shfl_sync(NSG_FULL, k, 31);
            const unsigned bal = __ballot_sync(NSG_FULL, keep);
            __syncwarp();
            if (keep) {
                const int o = w + __popc(bal & lanemask_lt());
                sk[o] = k;
                sp[o] = p;
            }
            w += __popc(bal);
            __syncwarp();
        }
        nk = w;
    }
    const int lo = sp[0];
    // move old entries i >= lo to i + #{r : sp[r] <= i}, top chunk first.  An
    // entry only moves up, so a chunk's writes land in chunks already read:
    // one barrier per chunk (between its reads and its writes) suffices.  Up
    // to 4 kept candidates (the common case) the count is 4 compares.
    const bool few = nk <= 4;
    const int p0 = sp[0], p1 = nk > 1 ? sp[1] : INT_MAX, p2 = nk > 2 ? sp[2] : INT_MAX,
              p3 = nk > 3 ? sp[3] : INT_MAX;
    for (int c = ((size - 1) >> 5) << 5; c >= (lo & ~31); c -= 32) {
        int i = c + (int)lane;
        uint64_t e = 0;
        int dst = cap;
        if (i >= lo && i < size) {
            e = list[i];
            dst = i + (few ? (p0 <= i) + (p1 <= i) + (p2 <= i) + (p3 <= i) : count_le(sp, nk, i));
        }
        __syncwarp();
        if (dst < cap) list[dst] = e;
    }
    for (int r = lane; r < nk; r += 32) {
        int f = sp[r] + r;
        if (f < cap) list[f] = sk[r];
    }
    size = min(size + nk, cap);
    __syncwarp();
    return lo < cap ? lo : cap;
}

}  // namespace nsg
