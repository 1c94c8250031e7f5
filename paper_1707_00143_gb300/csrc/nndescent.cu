// nndescent.cu -- approximate kNN graph by nn-descent (the approximate kNN
// graph the build starts from, Section 3.5 (ii); Dong, Charikar and Li's
// method, which the paper uses for its million-scale builds).
//
// The published method made deterministic and synchronous, so that the GPU
// result is a function of the inputs alone:
//   init     node v's list: the first K distinct ids != v among
//            splitmix64(seed + v * 0x9e3779b97f4a7c15 + t) mod n, t = 0, 1, ...,
//            all flagged new (key = (d2, id); "old" is bit 31 of the id word);
//   sample   newS(v) = the first S new entries (key order), oldS(v) = the first
//            S old ones; the sampled new entries become old;
//   reverse  rnew(u) = the Sr smallest keys (d(u, v), v) over {v : u in newS(v)}
//            (rold likewise over oldS), from a CSR of all reverse pairs;
//   join     NEW(v) = newS u rnew, OLD(v) = (oldS u rold) \ NEW.  The local
//            join offers every q in NEW(v) u OLD(v) to every p in NEW(v) and p
//            to q; node p therefore receives NEW(v) u OLD(v) for every v with
//            p in NEW(v) and NEW(v) for every v with p in OLD(v).  One warp per
//            p gathers those (a membership CSR), measures the ones its visited
//            set has not seen, and keeps the K smallest keys of its list and
//            the offers (new entries flagged new);
//   stop     after `iters` iterations, or once an iteration changes at most
//            delta * n * K list entries.
// Each step reads only what the previous step wrote, so the result does not
// depend on the order in which warps or atomics run.
#include <algorithm>

#include "kernels.h"
#include "lowp.cuh"
#include "search_core.cuh"

namespace nsg {
namespace {

constexpr int ND_W = 64;      // candidate batch per warp
constexpr int ND_HASH = 1024; // visited slots per warp in the join

__device__ __forceinline__ uint64_t nd_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Per-warp shared memory: list [K], first [K] (the list at the iteration's
// start), batch keys / merge scratch [ND_W], ids / positions [ND_W], hash.
struct NdSmem {
    uint64_t *list, *first, *keys, *ck, *sk;
    int *ids, *cp, *sp;
    uint32_t *hash;
};

__host__ __device__ inline size_t nd_warp_bytes(int K) {
    return 8ull * (2 * K + 3 * ND_W) + 4ull * (3 * ND_W + ND_HASH);
}

__device__ inline NdSmem nd_carve(unsigned char *p, int K) {
    NdSmem s;
    s.hash = reinterpret_cast<uint32_t *>(p);
    s.list = reinterpret_cast<uint64_t *>(s.hash + ND_HASH);
    s.first = s.list + K;
    s.keys = s.first + K;
    s.ck = s.keys + ND_W;
    s.sk = s.ck + ND_W;
    s.ids = reinterpret_cast<int *>(s.sk + ND_W);
    s.cp = s.ids + ND_W;
    s.sp = s.cp + ND_W;
    return s;
}

struct NdArgs {
    const float4 *base4;
    int dp4;
    int64_t n;
    int K, S, Sr;
    uint64_t seed;
    uint64_t *lists;  // [n][K] keys, bit 31 of the id word = old
    uint64_t *newS, *oldS;  // [n][S] sampled keys (their d2 is d(v, u))
    int *nnew, *nold;       // [n]
    int *rcnt_new, *rcnt_old;      // [n] reverse-pair counts, then fill cursors
    const int64_t *roff_new, *roff_old;  // [n + 1] CSR offsets
    uint64_t *rpair_new, *rpair_old;     // reverse pairs: (d2 << 32) | v
    int *NEWs, *OLDs;       // [n][S + Sr] join sets
    int *cNEW, *cOLD;       // [n]
    int *mcnt;              // [n] membership counts, then fill cursors
    const int64_t *moff;    // [n + 1]
    int *members;           // (v << 1) | (p in NEW(v))
    unsigned long long *updates;
    // 8-bit copy (rows of dc 16-byte chunks, x - lo) when it holds every
    // distance exactly, else nullptr: distances on FP32 rows
    const uint4 *u8;
    int dc, d;
    float lo;
};

// The distance functor for node v's row as the query: FP32 rows, or the exact
// 8-bit copy (a quarter of the bytes, the same keys), laid out as the 8-bit
// search form lays it out (lanes of 2 16-byte chunks, 3 row groups in flight;
// 8 for rows of 513..1024 values).
template <int G, int V, int U, bool U8, class F>
__device__ __forceinline__ void nd_with_dist(const NdArgs &a, int64_t v, F &&f) {
    if constexpr (U8) {
        constexpr int VG = V * G;
        constexpr int G8 = VG / 8 < 1 ? 1 : (VG / 8 > 32 ? 32 : VG / 8);
        constexpr int VC = VG / (4 * G8);
        constexpr int R8 = V == 8 ? 8 : (V > 8 ? 2 : 3);
        DistU8<G8, VC, R8> dist{{}, a.u8, a.dc};
        dist.Q.load(reinterpret_cast<const float *>(a.base4 + v * a.dp4), a.d, a.lo, 1.0f);
        f(dist);
    } else {
        DistF32<G, V, U> dist{{}, a.base4, a.dp4};
        dist.Q.load_row(a.base4 + v * a.dp4, a.dp4);
        f(dist);
    }
}

// init: K distinct seeded random neighbours per node, sorted by key.  One warp
// per node: lane 0 draws, the warp checks each draw against the ids so far.
template <int G, int V, int U, bool U8>
__global__ void __launch_bounds__(128) nd_init_kernel(NdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    NdSmem s = nd_carve(smem + warp * ((nd_warp_bytes(a.K) + 15) & ~size_t(15)), a.K);
    int *got = reinterpret_cast<int *>(s.first);  // K ids (the first-list space is free here)
    for (int64_t v = (int64_t)blockIdx.x * wpb + warp; v < a.n; v += (int64_t)gridDim.x * wpb) {
        int m = 0;
        for (uint64_t t = 0; m < a.K; ++t) {
            const int x = (int)(nd_splitmix64(a.seed + (uint64_t)v * 0x9e3779b97f4a7c15ull + t) % (uint64_t)a.n);
            bool dup = x == (int)v;
            for (int b = 0; b < m; b += 32) {
                const int j = b + (int)lane;
                dup |= __any_sync(NSG_FULL, j < m && got[j] == x);
            }
            if (!dup) {
                if (lane == 0) got[m] = x;
                __syncwarp();
                ++m;
            }
        }
        int size = 0;
        nd_with_dist<G, V, U, U8>(a, v, [&](const auto &dist) {
            for (int c0 = 0; c0 < a.K; c0 += ND_W) {
                const int cnt = min(ND_W, a.K - c0);
                for (int j = lane; j < cnt; j += 32) s.ids[j] = got[c0 + j];
                __syncwarp();
                dist(s.ids, cnt, s.keys);
                warp_merge(s.list, a.K, size, s.keys, cnt, s.ck, s.cp, s.sk, s.sp);
            }
        });
        for (int j = lane; j < a.K; j += 32) a.lists[v * a.K + j] = s.list[j];  // all new
        __syncwarp();
    }
}

// sample: newS / oldS in key order, sampled new entries marked old; reverse
// pairs counted per target.
__global__ void nd_sample_kernel(NdArgs a) {
    const unsigned lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < a.n; v += warps) {
        int cn = 0, co = 0;
        for (int b = 0; b < a.K; b += 32) {
            const int j = b + (int)lane;
            const uint64_t e = j < a.K ? a.lists[v * a.K + j] : 0;
            const bool isnew = j < a.K && !(e & CHK), isold = j < a.K && (e & CHK);
            const unsigned bn = __ballot_sync(NSG_FULL, isnew), bo = __ballot_sync(NSG_FULL, isold);
            const int rn = cn + __popc(bn & lanemask_lt()), ro = co + __popc(bo & lanemask_lt());
            if (isnew && rn < a.S) {
                a.newS[v * a.S + rn] = e;
                a.lists[v * a.K + j] = e | CHK;
                atomicAdd(&a.rcnt_new[kid(e)], 1);
            }
            if (isold && ro < a.S) {
                a.oldS[v * a.S + ro] = kval(e);
                atomicAdd(&a.rcnt_old[kid(e)], 1);
            }
            cn += __popc(bn);
            co += __popc(bo);
        }
        if (lane == 0) {
            a.nnew[v] = min(cn, a.S);
            a.nold[v] = min(co, a.S);
        }
    }
}

// reverse pairs into the CSR (order inside a segment is arbitrary: only the
// segment's smallest keys are used)
__global__ void nd_reverse_fill_kernel(NdArgs a) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.n * a.S;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = x / a.S;
        const int i = (int)(x - v * a.S);
        if (i < a.nnew[v]) {
            const uint64_t e = a.newS[x];
            const int u = kid(e);
            const int64_t pos = a.roff_new[u] + atomicAdd(&a.rcnt_new[u], 1);
            a.rpair_new[pos] = (e & 0xffffffff00000000ull) | (uint32_t)v;
        }
        if (i < a.nold[v]) {
            const uint64_t e = a.oldS[x];
            const int u = kid(e);
            const int64_t pos = a.roff_old[u] + atomicAdd(&a.rcnt_old[u], 1);
            a.rpair_old[pos] = (e & 0xffffffff00000000ull) | (uint32_t)v;
        }
    }
}

// The Sr smallest keys of a CSR segment: ids written to out[0..cnt).
__device__ void nd_topk_segment(const uint64_t *seg, int64_t len, int Sr, NdSmem &s, int *out, int *cnt) {
    const unsigned lane = lane_id();
    int size = 0;
    if (Sr < 1) len = 0;
    for (int64_t c0 = 0; c0 < len; c0 += ND_W) {
        const int m = len - c0 < ND_W ? (int)(len - c0) : ND_W;
        for (int j = lane; j < m; j += 32) s.keys[j] = seg[c0 + j];
        __syncwarp();
        warp_merge(s.list, Sr, size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
    }
    for (int j = lane; j < size; j += 32) out[j] = kid(s.list[j]);
    if (lane == 0) *cnt = size;
    __syncwarp();
}

// join sets: NEW(v) = newS u rnew, OLD(v) = (oldS u rold) \ NEW; membership counted.
__global__ void __launch_bounds__(128) nd_sets_kernel(NdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    NdSmem s = nd_carve(smem + warp * ((nd_warp_bytes(a.K) + 15) & ~size_t(15)), a.K);
    const int W2 = a.S + a.Sr;
    int *rn = reinterpret_cast<int *>(s.first);  // Sr ids each
    int *ro = rn + a.Sr;
    for (int64_t v = (int64_t)blockIdx.x * wpb + warp; v < a.n; v += (int64_t)gridDim.x * wpb) {
        int crn = 0, cro = 0;
        nd_topk_segment(a.rpair_new + a.roff_new[v], a.roff_new[v + 1] - a.roff_new[v], a.Sr, s, rn, &crn);
        crn = __shfl_sync(NSG_FULL, crn, 0);
        nd_topk_segment(a.rpair_old + a.roff_old[v], a.roff_old[v + 1] - a.roff_old[v], a.Sr, s, ro, &cro);
        cro = __shfl_sync(NSG_FULL, cro, 0);
        int *NEW = a.NEWs + v * W2;
        int *OLD = a.OLDs + v * W2;
        // candidate lists in order: newS, rnew | oldS, rold; a later copy of an id is dropped
        const int nn = a.nnew[v], no = a.nold[v];
        int cN = 0, cO = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const int len = pass == 0 ? nn + crn : no + cro;
            for (int b = 0; b < len; b += 32) {
                const int j = b + (int)lane;
                int x = -1;
                if (j < len) {
                    if (pass == 0) x = j < nn ? kid(a.newS[v * a.S + j]) : rn[j - nn];
                    else x = j < no ? kid(a.oldS[v * a.S + j]) : ro[j - no];
                }
                bool keep = x >= 0;
                // not in NEW so far, not earlier in this chunk, not in OLD so far
                for (int t = 0; t < cN && keep; ++t) keep = NEW[t] != x;
                if (pass == 1)
                    for (int t = 0; t < cO && keep; ++t) keep = OLD[t] != x;
                // earlier lanes of this chunk with the same id
                const unsigned same = __match_any_sync(NSG_FULL, x);
                keep = keep && (same & lanemask_lt()) == 0;
                const unsigned bal = __ballot_sync(NSG_FULL, keep);
                const int r = __popc(bal & lanemask_lt());
                if (keep) {
                    if (pass == 0) NEW[cN + r] = x;
                    else OLD[cO + r] = x;
                }
                if (pass == 0) cN += __popc(bal);
                else cO += __popc(bal);
                __syncwarp();
            }
        }
        for (int j = lane; j < cN; j += 32) atomicAdd(&a.mcnt[NEW[j]], 1);
        for (int j = lane; j < cO; j += 32) atomicAdd(&a.mcnt[OLD[j]], 1);
        if (lane == 0) {
            a.cNEW[v] = cN;
            a.cOLD[v] = cO;
        }
        __syncwarp();
    }
}

__global__ void nd_member_fill_kernel(NdArgs a) {
    const int W2 = a.S + a.Sr;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.n * W2;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = x / W2;
        const int i = (int)(x - v * W2);
        if (i < a.cNEW[v]) {
            const int p = a.NEWs[x];
            a.members[a.moff[p] + atomicAdd(&a.mcnt[p], 1)] = (int)(v << 1) | 1;
        }
        if (i < a.cOLD[v]) {
            const int p = a.OLDs[x];
            a.members[a.moff[p] + atomicAdd(&a.mcnt[p], 1)] = (int)(v << 1);
        }
    }
}

// The offers to p (NEW(v) u OLD(v) for members v with p in NEW(v), NEW(v)
// for the others), the ones the visited set has not seen measured, and p's
// list cut to its K smallest keys of itself and them.
template <int G, int V, int U, bool U8>
__global__ void __launch_bounds__(128) nd_join_kernel(NdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    NdSmem s = nd_carve(smem + warp * ((nd_warp_bytes(a.K) + 15) & ~size_t(15)), a.K);
    const uint32_t hmask = ND_HASH - 1;
    const int hshift = 32 - 10;  // log2(ND_HASH)
    const int W2 = a.S + a.Sr;
    for (int64_t p = (int64_t)blockIdx.x * wpb + warp; p < a.n; p += (int64_t)gridDim.x * wpb) {
        hash_clear(s.hash, ND_HASH);
        for (int j = lane; j < a.K; j += 32) {
            const uint64_t e = a.lists[p * a.K + j];
            s.list[j] = e;
            s.first[j] = kval(e);
            visit(s.hash, hmask, hshift, kid(e));  // the list's own ids need no offer
        }
        __syncwarp();
        if (lane == 0) visit(s.hash, hmask, hshift, (int)p);
        __syncwarp();
        int size = a.K;
        nd_with_dist<G, V, U, U8>(a, p, [&](const auto &dist) {
            int m = 0;
            const int64_t m0 = a.moff[p], m1 = a.moff[p + 1];
            for (int64_t mi = m0; mi < m1; ++mi) {
                const int tag = a.members[mi];
                const int64_t v = tag >> 1;
                const int cn = a.cNEW[v], co = (tag & 1) ? a.cOLD[v] : 0;
                for (int b = 0; b < cn + co; b += 32) {
                    const int j = b + (int)lane;
                    const int x = j < cn ? a.NEWs[v * W2 + j] : (j < cn + co ? a.OLDs[v * W2 + j - cn] : -1);
                    // p itself is among its own offers (p is in NEW(v)); the visited set
                    // may have forgotten it, so it is excluded by id
                    const bool fresh = x >= 0 && x != (int)p && visit(s.hash, hmask, hshift, x);
                    const unsigned bal = __ballot_sync(NSG_FULL, fresh);
                    const int cnt = __popc(bal);
                    if (m + cnt > ND_W) {  // flush the batch first
                        __syncwarp();
                        dist(s.ids, m, s.keys);
                        warp_merge(s.list, a.K, size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
                        m = 0;
                    }
                    if (fresh) s.ids[m + __popc(bal & lanemask_lt())] = x;
                    m += cnt;
                    __syncwarp();
                }
            }
            if (m > 0) {
                dist(s.ids, m, s.keys);
                warp_merge(s.list, a.K, size, s.keys, m, s.ck, s.cp, s.sk, s.sp);
            }
        });
        // entries that were not in the list at the iteration's start
        int changed = 0;
        for (int j = lane; j < a.K; j += 32) {
            const uint64_t k = kval(s.list[j]);
            int lo = 0, hi = a.K;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s.first[mid] < k) lo = mid + 1;
                else hi = mid;
            }
            changed += !(lo < a.K && s.first[lo] == k);
            a.lists[p * a.K + j] = s.list[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) changed += __shfl_xor_sync(NSG_FULL, changed, o);
        if (lane == 0 && changed) atomicAdd(a.updates, (unsigned long long)changed);
        __syncwarp();
    }
}

// the lists as ids and distances (key order)
__global__ void nd_export_kernel(const uint64_t *lists, int64_t total, int *ids, float *d2) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t e = lists[x];
        ids[x] = kid(e);
        if (d2) d2[x] = kd2(e);
    }
}

// Exclusive prefix sum of cnt[0..n) into off[0..n] (off[n] = total), three
// passes: per-block sums, one block over the block sums, per-block offsets.
constexpr int SCAN_T = 1024, SCAN_PER = 4;

__global__ void scan_blocks_kernel(const int *cnt, int64_t n, int64_t *off, int64_t *bsum) {
    __shared__ int64_t t[SCAN_T];
    const int64_t base = (int64_t)blockIdx.x * SCAN_T * SCAN_PER;
    int64_t loc[SCAN_PER], run = 0;
    for (int e = 0; e < SCAN_PER; ++e) {
        const int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + e;
        loc[e] = run;
        run += i < n ? cnt[i] : 0;
    }
    t[threadIdx.x] = run;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {  // inclusive scan of the thread sums
        const int64_t x = threadIdx.x >= (unsigned)o ? t[threadIdx.x - o] : 0;
        __syncthreads();
        t[threadIdx.x] += x;
        __syncthreads();
    }
    const int64_t before = threadIdx.x ? t[threadIdx.x - 1] : 0;
    for (int e = 0; e < SCAN_PER; ++e) {
        const int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + e;
        if (i < n) off[i] = before + loc[e];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = t[SCAN_T - 1];
}

__global__ void scan_sums_kernel(int64_t *bsum, int nb, int64_t *off, int64_t n) {
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t x = bsum[b];
        bsum[b] = run;
        run += x;
    }
    off[n] = run;
}

__global__ void scan_add_kernel(int64_t *off, int64_t n, const int64_t *bsum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += bsum[i / (SCAN_T * SCAN_PER)];
}

cudaError_t exclusive_scan(const int *cnt, int64_t n, int64_t *off, int64_t *bsum, cudaStream_t st) {
    const int nb = (int)((n + SCAN_T * SCAN_PER - 1) / (SCAN_T * SCAN_PER));
    scan_blocks_kernel<<<nb, SCAN_T, 0, st>>>(cnt, n, off, bsum);
    scan_sums_kernel<<<1, 32, 0, st>>>(bsum, nb, off, n);
    scan_add_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(off, n, bsum);
    return cudaGetLastError();
}

int grid_for(int64_t units, int per_block) {
    const int64_t b = (units + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 32));
}

template <typename Kern>
cudaError_t warp_launch(Kern k, const NdArgs &a, size_t per_warp, cudaStream_t st) {
    const int wpb = 4;
    const size_t smem = per_warp * wpb;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid_for(a.n, wpb), wpb * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t nndescent_scratch_bytes(int64_t n, int K, int S, int Sr) {
    const int64_t W2 = S + Sr;
    const int64_t nb = (n + SCAN_T * SCAN_PER - 1) / (SCAN_T * SCAN_PER);
    return (size_t)(8 * n * K                 // lists
                    + 2 * 8 * n * S           // newS, oldS
                    + 2 * 4 * n               // nnew, nold
                    + 2 * 4 * n               // reverse counts
                    + 2 * 8 * (n + 1)         // reverse offsets
                    + 2 * 8 * n * S           // reverse pairs
                    + 2 * 4 * n * W2          // NEW, OLD
                    + 2 * 4 * n               // their counts
                    + 4 * n + 8 * (n + 1)     // membership counts, offsets
                    + 4 * 2 * n * W2          // members
                    + 8 * nb + 8              // scan block sums, updates
                    + 16 * 32);               // alignment slack
}

cudaError_t launch_nndescent(const NnDescentLaunch &l, cudaStream_t st) {
    // the reverse samples are selected in the space of one list (Sr <= K)
    if (l.n < 2 || l.K < 1 || l.K >= l.n || l.S < 0 || l.Sr < 0 || l.Sr > l.K || !l.scratch)
        return cudaErrorInvalidValue;
    const int64_t n = l.n;
    const int K = l.K, S = l.S, Sr = l.Sr, W2 = S + Sr;
    unsigned char *p = static_cast<unsigned char *>(l.scratch);
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += (bytes + 15) & ~size_t(15);
        return q;
    };
    NdArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.dp4 = l.dp / 4;
    a.n = n;
    a.K = K;
    a.S = S;
    a.Sr = Sr;
    a.seed = l.seed;
    a.u8 = reinterpret_cast<const uint4 *>(l.u8);
    a.dc = l.u8_chunks;
    a.d = l.d;
    a.lo = l.u8_lo;
    a.lists = reinterpret_cast<uint64_t *>(take(8ull * n * K));
    a.newS = reinterpret_cast<uint64_t *>(take(8ull * n * std::max(S, 1)));
    a.oldS = reinterpret_cast<uint64_t *>(take(8ull * n * std::max(S, 1)));
    a.nnew = reinterpret_cast<int *>(take(4ull * n));
    a.nold = reinterpret_cast<int *>(take(4ull * n));
    a.rcnt_new = reinterpret_cast<int *>(take(4ull * n));
    a.rcnt_old = reinterpret_cast<int *>(take(4ull * n));
    int64_t *roff_new = reinterpret_cast<int64_t *>(take(8ull * (n + 1)));
    int64_t *roff_old = reinterpret_cast<int64_t *>(take(8ull * (n + 1)));
    a.roff_new = roff_new;
    a.roff_old = roff_old;
    a.rpair_new = reinterpret_cast<uint64_t *>(take(8ull * n * std::max(S, 1)));
    a.rpair_old = reinterpret_cast<uint64_t *>(take(8ull * n * std::max(S, 1)));
    a.NEWs = reinterpret_cast<int *>(take(4ull * n * std::max(W2, 1)));
    a.OLDs = reinterpret_cast<int *>(take(4ull * n * std::max(W2, 1)));
    a.cNEW = reinterpret_cast<int *>(take(4ull * n));
    a.cOLD = reinterpret_cast<int *>(take(4ull * n));
    a.mcnt = reinterpret_cast<int *>(take(4ull * n));
    int64_t *moff = reinterpret_cast<int64_t *>(take(8ull * (n + 1)));
    a.moff = moff;
    a.members = reinterpret_cast<int *>(take(4ull * 2 * n * std::max(W2, 1)));
    const int64_t nb = (n + SCAN_T * SCAN_PER - 1) / (SCAN_T * SCAN_PER);
    int64_t *bsum = reinterpret_cast<int64_t *>(take(8ull * nb));
    a.updates = reinterpret_cast<unsigned long long *>(take(8));
    const size_t per_warp = (nd_warp_bytes(K) + 15) & ~size_t(15);
    cudaError_t e = cudaSuccess;
    const int dp4 = a.dp4;
    const bool u8 = a.u8 != nullptr;
    NSG_DISPATCH_DP4(dp4, {
        e = u8 ? warp_launch(nd_init_kernel<G_, V_, U_, true>, a, per_warp, st)
               : warp_launch(nd_init_kernel<G_, V_, U_, false>, a, per_warp, st);
    });
    if (e != cudaSuccess) return e;
    int it = 0;
    unsigned long long upd = 0;
    const double stop_at = (double)l.delta * (double)n * (double)K;
    for (; it < l.iters; ++it) {
        if ((e = cudaMemsetAsync(a.rcnt_new, 0, 4ull * n, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.rcnt_old, 0, 4ull * n, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.mcnt, 0, 4ull * n, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.updates, 0, 8, st)) != cudaSuccess) return e;
        nd_sample_kernel<<<grid_for(n, 8), 256, 0, st>>>(a);
        if ((e = exclusive_scan(a.rcnt_new, n, roff_new, bsum, st)) != cudaSuccess) return e;
        if ((e = exclusive_scan(a.rcnt_old, n, roff_old, bsum, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.rcnt_new, 0, 4ull * n, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.rcnt_old, 0, 4ull * n, st)) != cudaSuccess) return e;
        nd_reverse_fill_kernel<<<grid_for(n * std::max(S, 1), 256), 256, 0, st>>>(a);
        if ((e = warp_launch(nd_sets_kernel, a, per_warp, st)) != cudaSuccess) return e;
        if ((e = exclusive_scan(a.mcnt, n, moff, bsum, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.mcnt, 0, 4ull * n, st)) != cudaSuccess) return e;
        nd_member_fill_kernel<<<grid_for(n * std::max(W2, 1), 256), 256, 0, st>>>(a);
        NSG_DISPATCH_DP4(dp4, {
            e = u8 ? warp_launch(nd_join_kernel<G_, V_, U_, true>, a, per_warp, st)
                   : warp_launch(nd_join_kernel<G_, V_, U_, false>, a, per_warp, st);
        });
        if (e != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&upd, a.updates, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if ((double)upd <= stop_at) {
            ++it;
            break;
        }
    }
    if (l.iters_run) *l.iters_run = it;
    if (l.last_updates) *l.last_updates = (int64_t)upd;
    nd_export_kernel<<<grid_for(n * K, 256), 256, 0, st>>>(a.lists, n * K, l.ids, l.d2);
    return cudaGetLastError();
}

}  // namespace nsg
