// knn_tc.cu -- brute-force k nearest neighbours on the 5th-generation tensor
// cores (serial scan of Section 4.1.2; the kNN graph G of Alg. 2 and the
// ground truth of Eq. 1).
//
// d2(q, x) = |q|^2 + (|x|^2 - 2 q.x): the dot products are a BF16 GEMM with
// FP32 accumulation in TMEM (tcgen05.mma, M = 128 query rows per CTA, N = 128
// base rows per tile, operands staged by TMA with 128-byte swizzle).  On
// integer data in 0..255 with d <= 128 every product, partial sum, norm and
// the final combination is an integer below 2^24, so the distances are exact
// and the selection below equals the serial scan bit for bit; the launcher
// checks the data and reports "not applicable" otherwise.
//
// CTA = 6 warps: warp 0 issues TMA (the 128 x d query tile once, then a ring
// of base tiles), warp 1 owns TMEM and issues the MMAs into two accumulator
// buffers, warps 2-5 are the epilogue: thread r holds query row r's running
// top-k.  A base column j enters row r's candidate buffer only when
// |x_j|^2 - 2 q.x_j < (current k-th distance) - |q|^2; the common case costs
// one FMA and one min per element (a group of 16 columns is tested through its
// minimum).  Columns arrive in increasing id, so a strict comparison on the
// distance alone implements the (distance, id) order.  Buffers of 16+ keys are
// merged warp-cooperatively into the row's sorted list, which lives in the
// output arrays.
#include <algorithm>
#include <cstdlib>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace nsg {

namespace {

constexpr int TC_M = 128;       // query rows per CTA (TMEM lanes)
constexpr int TC_N = 128;       // base rows per tile (accumulator columns)
constexpr int TC_BOXK = 64;     // bf16 elements per 128-byte swizzle atom
constexpr int TC_BUF = 64;      // candidate buffer per row
constexpr int TC_MERGE_AT = 48; // merge when a buffer holds this many (+ 16 per test < 64)
constexpr int TC_THREADS = 192;
constexpr int TC_MAXK = 256;

struct TcArgs {
    const float *qn;  // [m] squared norms of the query rows
    const float *xn;  // [ntiles * 128] squared norms of the base rows
    int64_t m, n, q0;
    int self_join, KL;
    int t0, t1;       // base tiles [t0, t1) of this launch (one chunk of the base)
    int first, last;  // first chunk: lists start empty; last chunk: pad short lists
    int kb;  // 64-wide K chunks per row (streaming form)
    int *ids;
    float *d2;
    int *lsz;  // [m] list sizes carried between chunks
    int *err;
};

// DK = 64 or 128: the 128-row query tile stays in shared memory and a stage
// holds one base tile.  DK = 0: rows wider than 128 values; a stage holds one
// 64-wide K chunk of both the query tile and the base tile (16 KB each), and
// a tile takes dk/64 stages.
template <int DK>
struct TcCfg {
    static constexpr int KB = DK / TC_BOXK;                     // swizzle atoms along K (resident form)
    static constexpr int A_BYTES = TC_M * DK * 2;
    static constexpr int B_BYTES = DK ? TC_N * DK * 2 : 2 * TC_N * 128;  // one pipeline stage
    static constexpr int NS = DK == 64 ? 7 : (DK == 128 ? 3 : 4);       // stages
    static constexpr int OFF_B = A_BYTES;
    static constexpr int OFF_BUF = OFF_B + NS * B_BYTES;
    static constexpr int OFF_WARP = OFF_BUF + TC_M * TC_BUF * 8;
    // per epilogue warp: merge list, sorted buffer, base norms, k-th slot, and
    // 16 values per lane for the insertion path (column-major, conflict-free)
    static constexpr int WARP_BYTES = TC_MAXK * 8 + TC_BUF * 8 + TC_N * 4 + 16 + 16 * 32 * 4;
    static constexpr int OFF_BAR = OFF_WARP + 4 * WARP_BYTES;
    static constexpr int NBAR = 2 * NS + 6;  // a_full, b_full[NS], b_empty[NS], acc_full[2], acc_empty[2], drain
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16 + 1024;  // + alignment slack
};

// Bitonic sort of 64 keys held two per lane (index lane and lane + 32), ascending.
__device__ __forceinline__ void bitonic64(uint64_t &a, uint64_t &b, unsigned lane) {
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {  // partner in the same lane: index lane vs lane + 32 (k = 64: ascending)
                const uint64_t mn = a < b ? a : b, mx = a < b ? b : a;
                a = mn;
                b = mx;
            } else {
                const uint64_t oa = __shfl_xor_sync(NSG_FULL, a, j), ob = __shfl_xor_sync(NSG_FULL, b, j);
                const bool lower = (lane & j) == 0;
                const bool up_a = (lane & k) == 0, up_b = ((lane + 32) & k) == 0;
                const uint64_t mna = oa < a ? oa : a, mxa = oa < a ? a : oa;
                const uint64_t mnb = ob < b ? ob : b, mxb = ob < b ? b : ob;
                a = (lower == up_a) ? mna : mxa;
                b = (lower == up_b) ? mnb : mxb;
            }
        }
    }
}

__device__ __forceinline__ int count_less(const uint64_t *a, int len, uint64_t key) {
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Merge row `src`'s buffer (c <= 63 keys) into its sorted list of s keys
// (output arrays, capacity KL), warp-cooperatively: the list is read once
// (all loads issued before use), the buffer sorted, and every key written to
// its rank in the union.
__device__ __noinline__ void merge_row(int src, int row_local, int64_t row_g, int &cnt, int &lsize,
                                       float &thrp, float qn_r, const uint64_t *bufs, uint64_t *ls,
                                       uint64_t *sb, uint64_t *thr_slot, int *ids, float *d2, int KL) {
    const unsigned lane = lane_id();
    const int c = __shfl_sync(NSG_FULL, cnt, src);
    const int s = __shfl_sync(NSG_FULL, lsize, src);
    const int rl = __shfl_sync(NSG_FULL, row_local, src);
    const int64_t rg = __shfl_sync(NSG_FULL, row_g, src);
    int *oid = ids + rg * KL;
    float *od = d2 + rg * KL;
    float lv[TC_MAXK / 32];
    int li[TC_MAXK / 32];
#pragma unroll
    for (int t = 0; t < TC_MAXK / 32; ++t) {
        const int i = t * 32 + (int)lane;
        if (i < s) {
            lv[t] = od[i];
            li[t] = oid[i];
        }
    }
    uint64_t a = (int)lane < c ? bufs[rl * TC_BUF + lane] : ~0ull;
    uint64_t b = (int)lane + 32 < c ? bufs[rl * TC_BUF + 32 + lane] : ~0ull;
    bitonic64(a, b, lane);
    sb[lane] = a;
    sb[lane + 32] = b;
#pragma unroll
    for (int t = 0; t < TC_MAXK / 32; ++t) {
        const int i = t * 32 + (int)lane;
        if (i < s) ls[i] = make_key(lv[t], li[t]);
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < TC_MAXK / 32; ++t) {
        const int i = t * 32 + (int)lane;
        if (i < s) {
            const uint64_t key = ls[i];
            const int p = i + count_less(sb, c, key);
            if (p < KL) {
                od[p] = kd2(key);
                oid[p] = kid(key);
                if (p == KL - 1) *thr_slot = key;
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = (int)lane + 32 * h;
        const uint64_t key = h ? b : a;
        if (j < c) {
            const int p = j + count_less(ls, s, key);
            if (p < KL) {
                od[p] = kd2(key);
                oid[p] = kid(key);
                if (p == KL - 1) *thr_slot = key;
            }
        }
    }
    __syncwarp();
    if ((int)lane == src) {
        cnt = 0;
        lsize = s + c < KL ? s + c : KL;
        if (lsize == KL) thrp = kd2(*thr_slot) - qn_r;
    }
    __syncwarp();
}

template <int DK>
__global__ void __launch_bounds__(TC_THREADS, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    using Cfg = TcCfg<DK>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = smem;
    unsigned char *sB = smem + Cfg::OFF_B;
    uint64_t *bufs = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BUF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Cfg::OFF_BAR);
    uint64_t *a_full = bars;
    uint64_t *b_full = bars + 1;
    uint64_t *b_empty = bars + 1 + Cfg::NS;
    uint64_t *acc_full = bars + 1 + 2 * Cfg::NS;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + Cfg::NBAR);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *gerr = a.err;

    const int warp = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;

    if (threadIdx.x == 0) {
        tc::mbar_init(a_full, 1);
        for (int s = 0; s < Cfg::NS; ++s) {
            tc::mbar_init(b_full + s, 1);
            tc::mbar_init(b_empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(acc_full + b, 1);
            tc::mbar_init(acc_empty + b, 4);
        }
        tc::mbar_init(drain, 1);
        *abort = *gerr ? 1 : 0;  // another CTA already failed: do nothing
        tc::fence_barrier_init();
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 2 * TC_N);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const bool skip = *abort != 0;  // uniform: read after the barrier

    if (skip) {
        // nothing issued; fall through to TMEM release
    } else if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            if (DK) {
                tc::mbar_expect_tx(a_full, Cfg::A_BYTES);
                for (int kb = 0; kb < Cfg::KB; ++kb)
                    tc::tma_load_2d(sA + kb * (TC_M * 128), &tmA, a_full, kb * TC_BOXK, (int)row0);
            }
            const int per_tile = DK ? 1 : a.kb;  // stages per tile
            const int nt = a.t1 - a.t0;
            int issued = 0;
            for (int c = 0; c < nt * per_tile; ++c) {
                const int s = c % Cfg::NS, tl = c / per_tile, kc = c - tl * per_tile, t = a.t0 + tl;
                if (!tc::mbar_wait(b_empty + s, ((c / Cfg::NS) & 1) ^ 1, abort, gerr)) break;
                tc::mbar_expect_tx(b_full + s, Cfg::B_BYTES);
                unsigned char *dst = sB + s * Cfg::B_BYTES;
                if (DK) {
                    for (int kb = 0; kb < Cfg::KB; ++kb)
                        tc::tma_load_2d(dst + kb * (TC_N * 128), &tmB, b_full + s, kb * TC_BOXK, t * TC_N);
                } else {
                    tc::tma_load_2d(dst, &tmA, b_full + s, kc * TC_BOXK, (int)row0);
                    tc::tma_load_2d(dst + TC_M * 128, &tmB, b_full + s, kc * TC_BOXK, t * TC_N);
                }
                issued = c + 1;
            }
            if (*abort) {
                // drain: wait (bounded) for the copies still in flight
                volatile int local = 0;
                if (DK) tc::mbar_wait(a_full, 0, &local, nullptr);
                for (int c = issued - Cfg::NS < 0 ? 0 : issued - Cfg::NS; c < issued; ++c) {
                    local = 0;
                    tc::mbar_wait(b_full + c % Cfg::NS, (c / Cfg::NS) & 1, &local, nullptr);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
            const uint32_t a_base = tc::smem_u32(sA), b_base = tc::smem_u32(sB);
            bool ok = DK ? tc::mbar_wait(a_full, 0, abort, gerr) : true;
            const int per_tile = DK ? 1 : a.kb;
            int c = 0;
            for (int t = 0; ok && t < a.t1 - a.t0; ++t) {  // local tile index
                const int buf = t & 1;
                if (!tc::mbar_wait(acc_empty + buf, ((t >> 1) & 1) ^ 1, abort, gerr)) break;
                tc::fence_after_sync();
                for (int kc = 0; ok && kc < per_tile; ++kc, ++c) {
                    const int s = c % Cfg::NS;
                    if (!tc::mbar_wait(b_full + s, (c / Cfg::NS) & 1, abort, gerr)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    if (DK) {
#pragma unroll
                        for (int kk = 0; kk < (DK ? DK : 64) / 16; ++kk) {
                            const uint32_t koff = (kk >> 2) * (TC_M * 128) + (kk & 3) * 32;
                            const uint32_t boff = s * Cfg::B_BYTES + (kk >> 2) * (TC_N * 128) + (kk & 3) * 32;
                            tc::mma_bf16(tmem + buf * TC_N, tc::sdesc_sw128(a_base + koff),
                                         tc::sdesc_sw128(b_base + boff), idesc, kk > 0 ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t st = b_base + s * Cfg::B_BYTES + kk * 32;
                            tc::mma_bf16(tmem + buf * TC_N, tc::sdesc_sw128(st), tc::sdesc_sw128(st + TC_M * 128),
                                         idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(b_empty + s);
                }
                if (!ok) break;
                tc::mma_commit(acc_full + buf);
            }
            // every MMA issued so far has completed before TMEM is released
            tc::mma_commit(drain);
            volatile int local = 0;
            tc::mbar_wait(drain, 0, &local, nullptr);
        }
    } else {
        // ---------------- epilogue: warps 2..5 ----------------
        const int q = warp & 3;  // TMEM lane quadrant of this warp
        const int ew = warp - 2;
        unsigned char *wsm = smem + Cfg::OFF_WARP + ew * Cfg::WARP_BYTES;
        uint64_t *ls = reinterpret_cast<uint64_t *>(wsm);
        uint64_t *sb = ls + TC_MAXK;
        float *xs = reinterpret_cast<float *>(sb + TC_BUF);
        uint64_t *thr_slot = reinterpret_cast<uint64_t *>(xs + TC_N);
        float *tvs = reinterpret_cast<float *>(thr_slot + 2);  // [16][32]
        const int row_local = q * 32 + lane;
        const int64_t row_g = row0 + row_local;
        const bool valid = row_g < a.m;
        const float qn_r = valid ? a.qn[row_g] : 0.0f;
        const int64_t self_id = a.self_join ? a.q0 + row_g : -1;
        uint64_t *mybuf = bufs + row_local * TC_BUF;
        // the row's list (size and k-th key) carried over from earlier chunks;
        // a row past the end takes nothing: its threshold is -inf
        int cnt = 0, lsize = valid && !a.first ? a.lsz[row_g] : 0;
        float thrp = __int_as_float(valid ? 0x7f800000 : 0xff800000);
        if (valid && lsize == a.KL) thrp = a.d2[row_g * a.KL + a.KL - 1] - qn_r;
        const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
        bool ok = true;
        const float4 *xn4 = reinterpret_cast<const float4 *>(a.xn);
        float4 xnext = __ldg(xn4 + (int64_t)a.t0 * (TC_N / 4) + lane);  // norms one tile ahead
        for (int tl = 0; tl < a.t1 - a.t0; ++tl) {
            const int buf = tl & 1, t = a.t0 + tl;
            const int64_t col0 = (int64_t)t * TC_N;
            // columns jj < lim exist; jj == self_local is the row itself
            const int lim = a.n - col0 < TC_N ? (int)(a.n - col0) : TC_N;
            const int self_local = self_id >= col0 && self_id < col0 + TC_N ? (int)(self_id - col0) : -1;
            __syncwarp();
            reinterpret_cast<float4 *>(xs)[lane] = xnext;
            if (t + 1 < a.t1) xnext = __ldg(xn4 + (int64_t)(t + 1) * (TC_N / 4) + lane);
            __syncwarp();
            const bool got = tc::mbar_wait(acc_full + buf, (tl >> 1) & 1, abort, gerr);
            if (!__all_sync(NSG_FULL, got)) {  // warp-uniform before the .sync.aligned TMEM loads
                ok = false;
                break;
            }
            tc::fence_after_sync();
#pragma unroll 1
            for (int c = 0; c < TC_N / 32; ++c) {
                uint32_t v[32];
                tc::tmem_ld32(tq + buf * TC_N + c * 32, v);
                tc::tmem_ld_wait();
                if (c == TC_N / 32 - 1) {
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(acc_empty + buf);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // |x|^2 - 2 q.x for 16 columns and their minimum: one FMA
                    // and one min per element; the insertion path runs only
                    // when some column beats the row's current k-th distance
                    const int jb = c * 32 + h * 16;
                    const float4 *x4 = reinterpret_cast<const float4 *>(xs + jb);
                    float tv[16];
#pragma unroll
                    for (int j4 = 0; j4 < 4; ++j4) {
                        const float4 xv = x4[j4];
                        const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            tv[j4 * 4 + e] = fmaf(-2.0f, __uint_as_float(v[h * 16 + j4 * 4 + e]), xa[e]);
                    }
                    float m8[8];  // minimum as a tree (independent instructions)
#pragma unroll
                    for (int j = 0; j < 8; ++j) m8[j] = fminf(tv[2 * j], tv[2 * j + 1]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) m8[j] = fminf(m8[2 * j], m8[2 * j + 1]);
                    const float mn = fminf(fminf(m8[0], m8[1]), fminf(m8[2], m8[3]));
                    if (mn < thrp) {
                        // columns of this group that exist, are not the row itself, and
                        // beat the threshold: a bit mask, then one step per set bit
                        const int nv = lim - jb;
                        unsigned vm = nv >= 16 ? 0xffffu : (nv <= 0 ? 0u : (1u << nv) - 1u);
                        if ((unsigned)(self_local - jb) < 16u) vm &= ~(1u << (self_local - jb));
                        unsigned msk = 0;
#pragma unroll
                        for (int j = 0; j < 16; ++j) msk |= (tv[j] < thrp ? 1u : 0u) << j;
                        msk &= vm;
                        if (msk) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) tvs[j * 32 + lane] = tv[j];
                            while (msk) {
                                const int j = __ffs(msk) - 1;
                                msk &= msk - 1;
                                mybuf[cnt] = make_key(fmaxf(qn_r + tvs[j * 32 + lane], 0.0f), (int)(col0 + jb + j));
                                ++cnt;
                            }
                        }
                    }
                    unsigned need = __ballot_sync(NSG_FULL, cnt >= TC_MERGE_AT);
                    while (need) {
                        const int src = __ffs(need) - 1;
                        need &= need - 1;
                        merge_row(src, row_local, row_g, cnt, lsize, thrp, qn_r, bufs, ls, sb, thr_slot,
                                  a.ids, a.d2, a.KL);
                    }
                }
            }
        }
        if (ok) {
            unsigned need = __ballot_sync(NSG_FULL, cnt > 0);
            while (need) {
                const int src = __ffs(need) - 1;
                need &= need - 1;
                merge_row(src, row_local, row_g, cnt, lsize, thrp, qn_r, bufs, ls, sb, thr_slot, a.ids,
                          a.d2, a.KL);
            }
            if (!a.last) {  // carry the list size to the next chunk
                if (valid) a.lsz[row_g] = lsize;
            } else  // pad rows holding fewer than k candidates
            for (int src = 0; src < 32; ++src) {
                const int s = __shfl_sync(NSG_FULL, lsize, src);
                const int64_t rg = __shfl_sync(NSG_FULL, row_g, src);
                const bool v = __shfl_sync(NSG_FULL, valid ? 1 : 0, src);
                if (!v) continue;
                for (int i = s + lane; i < a.KL; i += 32) {
                    a.ids[rg * a.KL + i] = -1;
                    a.d2[rg * a.KL + i] = __int_as_float(0x7f800000);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (*abort && !skip && threadIdx.x == 0) atomicExch(a.err, 1);
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 2 * TC_N);
    }
}

// Row-wise BF16 copy with K padded to DK, squared norms of the rounded values,
// and a flag raised when a value is not an integer in 0..255.
__global__ void bf16_rows_kernel(const float *__restrict__ src, int64_t rows, int dp, __nv_bfloat16 *dst,
                                 int dk, float *norms, int64_t rows_pad, int *nonint) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned lane = lane_id();
    for (int64_t r = warp; r < rows_pad; r += nw) {
        float acc = 0.0f;
        bool bad = false;
        for (int c = lane; c < dk; c += 32) {
            float v = (r < rows && c < dp) ? src[r * dp + c] : 0.0f;
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            float hv = __bfloat162float(h);
            acc += hv * hv;
            bad |= !(v >= 0.0f && v <= 255.0f && v == rintf(v));
            if (r < rows) dst[r * dk + c] = h;
        }
        acc = group_sum<32>(acc);
        if (lane == 0) norms[r] = r < rows ? acc : 0.0f;
        if (__any_sync(NSG_FULL, bad) && lane == 0 && r < rows) atomicOr(nonint, 1);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D tensor map over a [rows][dk] bf16 matrix, box = 64 (K) x box_rows, 128B swizzle.
bool make_map(CUtensorMap *map, const void *ptr, int64_t rows, int dk, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dk, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dk * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BOXK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename T>
struct Scratch {
    T *p = nullptr;
    ~Scratch() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc(reinterpret_cast<void **>(&p), n * sizeof(T) + 16); }
};

}  // namespace

// Tensor-core kNN when the data allows an exact answer (integer 0..255,
// d <= 128, k <= 256); *used = 0 when it does not apply (nothing written).
cudaError_t launch_knn_tc(const KnnLaunch &l, int *used, cudaStream_t st) {
    *used = 0;
    if (l.nq <= 0 || l.k > TC_MAXK || l.dp > 1024 || !encode_fn()) return cudaSuccess;
    const int dk = l.dp <= 64 ? 64 : (l.dp <= 128 ? 128 : (l.dp + 63) / 64 * 64);
    const int64_t ntiles = (l.n + TC_N - 1) / TC_N;
    if (ntiles > INT32_MAX / TC_N) return cudaSuccess;
    const int64_t npad = ntiles * TC_N;
    Scratch<__nv_bfloat16> xb, qb;
    Scratch<float> xn, qn;
    Scratch<int> flag;
    cudaError_t e;
    if ((e = xb.alloc((size_t)l.n * dk)) != cudaSuccess) return e;
    if ((e = xn.alloc((size_t)npad)) != cudaSuccess) return e;
    if ((e = flag.alloc(2)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(flag.p, 0, 2 * sizeof(int), st)) != cudaSuccess) return e;
    const int grid_rows = sm_count() * 8;
    bf16_rows_kernel<<<grid_rows, 256, 0, st>>>(l.base, l.n, l.dp, xb.p, dk, xn.p, npad, flag.p);
    const __nv_bfloat16 *qsrc = xb.p + (l.self_join ? l.q0 * dk : 0);
    const float *qnorm = xn.p + (l.self_join ? l.q0 : 0);
    if (!l.self_join) {
        if ((e = qb.alloc((size_t)l.nq * dk)) != cudaSuccess) return e;
        if ((e = qn.alloc((size_t)l.nq)) != cudaSuccess) return e;
        bf16_rows_kernel<<<grid_rows, 256, 0, st>>>(l.queries, l.nq, l.dp, qb.p, dk, qn.p, l.nq, flag.p);
        qsrc = qb.p;
        qnorm = qn.p;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int h[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h, flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    // Integer data 0..255 with d <= 128: the GEMM-form distances are exact and
    // the k best lists are the answer.  Otherwise (float data, or wider rows
    // whose integer sums may pass 2^24) the GEMM keeps the KL = k + margin best
    // candidates by its BF16 distance and an exact FP32 re-rank picks the k.
    const bool exact = !h[0] && dk <= 128;
    const int KL = exact ? l.k : (l.k + (l.k / 2 > 32 ? l.k / 2 : 32) < TC_MAXK ? l.k + (l.k / 2 > 32 ? l.k / 2 : 32)
                                                                                 : TC_MAXK);
    if (!exact && KL < l.k + 16) return cudaSuccess;  // no room for a margin: exact scan instead
    CUtensorMap mA, mB;
    const int64_t arows = l.self_join ? l.n - l.q0 : l.nq;
    if (!make_map(&mA, qsrc, arows, dk, TC_M) || !make_map(&mB, xb.p, l.n, dk, TC_N)) return cudaSuccess;
    // the rows' sorted lists live in the output arrays (exact) or in scratch
    // (candidates); distances are kept even when the caller asked for ids only
    Scratch<float> d2s;
    Scratch<int> ids_s;
    float *d2out = l.d2;
    int *idsout = l.ids;
    if (!exact) {
        if ((e = ids_s.alloc((size_t)l.nq * KL)) != cudaSuccess) return e;
        idsout = ids_s.p;
    }
    if (!exact || !d2out) {
        if ((e = d2s.alloc((size_t)l.nq * KL)) != cudaSuccess) return e;
        d2out = d2s.p;
    }
    TcArgs a;
    a.qn = qnorm;
    a.xn = xn.p;
    a.m = l.nq;
    a.n = l.n;
    a.q0 = l.q0;
    a.self_join = l.self_join;
    a.KL = KL;
    a.kb = dk / TC_BOXK;
    a.ids = idsout;
    a.d2 = d2out;
    a.err = flag.p + 1;
    // The base is taken in chunks of ~48 MB of BF16 rows, one launch per chunk
    // over every query tile, so a chunk stays in L2 while all query tiles pass
    // over it (a single sweep per CTA would re-read a base larger than L2 from
    // HBM once per wave of CTAs).  Rows see columns in increasing id across
    // chunks, and their lists carry over through the output arrays and lsz.
    int64_t chunk_tiles = std::max<int64_t>(1, (int64_t(48) << 20) / ((int64_t)TC_N * dk * 2));
    if (const char *ct = getenv("NSG_KNN_CHUNK_TILES"))  // smaller chunks (tests)
        if (atoi(ct) > 0) chunk_tiles = atoi(ct);
    const int64_t nchunks = (ntiles + chunk_tiles - 1) / chunk_tiles;
    Scratch<int> lsz;
    if (nchunks > 1 && (e = lsz.alloc((size_t)l.nq)) != cudaSuccess) return e;
    a.lsz = lsz.p;
    const int64_t grid = (l.nq + TC_M - 1) / TC_M;
    for (int64_t c = 0; c < nchunks; ++c) {
        a.t0 = (int)(c * chunk_tiles);
        a.t1 = (int)std::min<int64_t>(ntiles, (c + 1) * chunk_tiles);
        a.first = c == 0;
        a.last = c == nchunks - 1;
        if (dk == 64) {
            auto kern = knn_tc_kernel<64>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<64>::SMEM)) !=
                cudaSuccess)
                return e;
            kern<<<(unsigned)grid, TC_THREADS, TcCfg<64>::SMEM, st>>>(mA, mB, a);
        } else if (dk == 128) {
            auto kern = knn_tc_kernel<128>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<128>::SMEM)) !=
                cudaSuccess)
                return e;
            kern<<<(unsigned)grid, TC_THREADS, TcCfg<128>::SMEM, st>>>(mA, mB, a);
        } else {
            auto kern = knn_tc_kernel<0>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<0>::SMEM)) !=
                cudaSuccess)
                return e;
            kern<<<(unsigned)grid, TC_THREADS, TcCfg<0>::SMEM, st>>>(mA, mB, a);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaMemcpyAsync(h, flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h[1]) return cudaErrorLaunchTimeout;  // a pipeline wait gave up (bounded waits)
    if (!exact) {
        if ((e = launch_knn_rerank(l, idsout, KL, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;  // scratch is freed on return
    }
    *used = 1;
    return cudaSuccess;
}

}  // namespace nsg
