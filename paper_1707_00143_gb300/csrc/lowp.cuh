// lowp.cuh -- traversal distances on low-precision copies of the base.
//
// Rows are stored as BF16 (8 values per 16-byte chunk), FP8-e4m3 (16 per
// chunk, values pre-multiplied by a per-tensor scale so the largest |x| maps
// to 448) or U8 (16 per chunk, integer arithmetic, below).  The query stays FP32 (scaled the same way), each chunk is widened
// to FP32 and the squared differences are accumulated in FP32.  Scaling all
// coordinates by one factor scales every squared distance by its square, so
// the traversal order is unaffected by it.  On integer data 0..255 the BF16
// copy is exact and so are its distances.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace nsg {

enum { PREC_F32 = 0, PREC_BF16 = 1, PREC_FP8 = 2, PREC_U8 = 3 };

// ---------------------------------------------------------------------------
// 8-bit integer form: x_u8 = clamp(rint((x - lo) * s), 0, 255), the query
// quantised the same way, squared differences summed exactly in int32 with
// __vabsdiffu4 (per-byte |a - b|) and __dp4a.  With lo = 0 and s = 1 (integer
// data 0..255) the copy, the query and every distance are exact, so the keys
// equal the FP32 keys while a row is a quarter of the FP32 bytes.
// ---------------------------------------------------------------------------
template <int G, int VC>
struct RowQueryU8 {
    uint4 q[VC];  // 16 quantised values per chunk
    // Returns (warp-uniform) whether the 8-bit map kept every query value.
    __device__ __forceinline__ bool load(const float *__restrict__ src, int d, float lo, float s) {
        const int sub = lane_id() % G;
        bool exact = true;
#pragma unroll
        for (int t = 0; t < VC; ++t) {
            uint32_t w[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                uint32_t word = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = (t * G + sub) * 16 + b * 4 + e;
                    const float y = j < d ? (__ldg(src + j) - lo) * s : 0.0f;
                    const float v = fminf(fmaxf(rintf(y), 0.0f), 255.0f);
                    exact &= v == y;
                    word |= (uint32_t)v << (8 * e);
                }
                w[b] = word;
            }
            q[t] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        return __all_sync(NSG_FULL, exact);
    }
};

template <int G, int VC, int U>
struct DistU8 {
    RowQueryU8<G, VC> Q;
    const uint4 *base;  // [n][dc] chunks of 16 bytes
    int dc;
    __device__ __forceinline__ void operator()(const int *ids, int m, uint64_t *keys) const {
        constexpr int PG = 32 / G;
        const int lane = lane_id(), grp = lane / G, sub = lane % G;
        for (int c0 = 0; c0 < m; c0 += PG * U) {
            uint4 x[U][VC];
            int id[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * PG + grp;
                id[u] = c < m ? ids[c] : -1;
                const uint4 *row = base + (int64_t)(id[u] < 0 ? 0 : id[u]) * dc;
#pragma unroll
                for (int t = 0; t < VC; ++t) {
                    const int k = t * G + sub;
                    x[u][t] = (id[u] >= 0 && k < dc) ? __ldg(row + k) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                unsigned s = 0;
#pragma unroll
                for (int t = 0; t < VC; ++t) {
                    const uint32_t a[4] = {x[u][t].x, x[u][t].y, x[u][t].z, x[u][t].w};
                    const uint32_t b[4] = {Q.q[t].x, Q.q[t].y, Q.q[t].z, Q.q[t].w};
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const unsigned df = __vabsdiffu4(a[w], b[w]);
                        s = __dp4a(df, df, s);
                    }
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(NSG_FULL, s, o, G);
                const int c = c0 + u * PG + grp;
                if (sub == 0 && c < m) keys[c] = make_key((float)s, id[u]);
            }
        }
        __syncwarp();
    }
    __device__ __forceinline__ void prefetch(const int *, int) const {}  // measured: no gain
    // every row, ahead of a gather that comes later
    __device__ __forceinline__ void prefetch_all(const int *ids, int m) const {
        prefetch_rows_l2(base, dc * 16, ids, m);
    }
    // staged gathers: the register gather's arithmetic on a shared-memory row
    __device__ __forceinline__ const void *row_addr(int id) const { return base + (int64_t)id * dc; }
    __device__ __forceinline__ int row_bytes() const { return dc * 16; }
    __device__ __forceinline__ float row_smem(const unsigned char *row) const {
        const uint4 *r = reinterpret_cast<const uint4 *>(row);
        const int sub = lane_id() % G;
        unsigned s = 0;
#pragma unroll
        for (int t = 0; t < VC; ++t) {
            const int k = t * G + sub;
            const uint4 x = k < dc ? r[k] : make_uint4(0, 0, 0, 0);
            const uint32_t a[4] = {x.x, x.y, x.z, x.w};
            const uint32_t b[4] = {Q.q[t].x, Q.q[t].y, Q.q[t].z, Q.q[t].w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const unsigned df = __vabsdiffu4(a[w], b[w]);
                s = __dp4a(df, df, s);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(NSG_FULL, s, o, G);
        return (float)s;
    }
};

template <int P>
struct PrecEpc;  // values per 16-byte chunk
template <>
struct PrecEpc<PREC_BF16> {
    static constexpr int value = 8;
};
template <>
struct PrecEpc<PREC_FP8> {
    static constexpr int value = 16;
};

__device__ __forceinline__ void unpack_bf16(const uint4 &c, float (&f)[8]) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

__device__ __forceinline__ void unpack_fp8(const uint4 &c, float (&f)[16]) {
    const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> (16 * h)), __NV_E4M3);
            float2 v = __half22float2(*reinterpret_cast<__half2 *>(&r));
            f[4 * i + 2 * h] = v.x;
            f[4 * i + 2 * h + 1] = v.y;
        }
    }
}

template <int P>
__device__ __forceinline__ void unpack(const uint4 &c, float (&f)[PrecEpc<P>::value]) {
    if constexpr (P == PREC_BF16) unpack_bf16(c, f);
    else unpack_fp8(c, f);
}

// Lane `sub` of a G-lane group holds chunks t*G + sub (t < VC) of the query.
template <int P, int G, int VC>
struct RowQueryLp {
    static constexpr int EPC = PrecEpc<P>::value;
    float q[VC][EPC];
    __device__ __forceinline__ void load(const float *__restrict__ src, int d, float scale) {
        const int sub = lane_id() % G;
#pragma unroll
        for (int t = 0; t < VC; ++t)
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
                const int j = (t * G + sub) * EPC + e;
                q[t][e] = j < d ? __ldg(src + j) * scale : 0.0f;
            }
    }
};

template <int P, int G, int VC, int U>
struct DistLp {
    static constexpr int EPC = PrecEpc<P>::value;
    RowQueryLp<P, G, VC> Q;
    const uint4 *base;  // [n][dc] chunks
    int dc;
    __device__ __forceinline__ void operator()(const int *ids, int m, uint64_t *keys) const {
        constexpr int PG = 32 / G;
        const int lane = lane_id(), grp = lane / G, sub = lane % G;
        for (int c0 = 0; c0 < m; c0 += PG * U) {
            uint4 x[U][VC];
            int id[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c = c0 + u * PG + grp;
                id[u] = c < m ? ids[c] : -1;
                const uint4 *row = base + (int64_t)(id[u] < 0 ? 0 : id[u]) * dc;
#pragma unroll
                for (int t = 0; t < VC; ++t) {
                    const int k = t * G + sub;
                    x[u][t] = (id[u] >= 0 && k < dc) ? __ldg(row + k) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float s = 0.0f;
#pragma unroll
                for (int t = 0; t < VC; ++t) {
                    float f[EPC];
                    unpack<P>(x[u][t], f);
#pragma unroll
                    for (int e = 0; e < EPC; ++e) {
                        const float df = f[e] - Q.q[t][e];
                        s = fmaf(df, df, s);
                    }
                }
                s = group_sum<G>(s);
                const int c = c0 + u * PG + grp;
                if (sub == 0 && c < m) keys[c] = make_key(s, id[u]);
            }
        }
        __syncwarp();
    }
    __device__ __forceinline__ void prefetch(const int *, int) const {}  // measured: no gain
    // every row, ahead of a gather that comes later
    __device__ __forceinline__ void prefetch_all(const int *ids, int m) const {
        prefetch_rows_l2(base, dc * 16, ids, m);
    }
    // staged gathers: the register gather's arithmetic on a shared-memory row
    __device__ __forceinline__ const void *row_addr(int id) const { return base + (int64_t)id * dc; }
    __device__ __forceinline__ int row_bytes() const { return dc * 16; }
    __device__ __forceinline__ float row_smem(const unsigned char *row) const {
        const uint4 *r = reinterpret_cast<const uint4 *>(row);
        const int sub = lane_id() % G;
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < VC; ++t) {
            const int k = t * G + sub;
            float f[EPC];
            unpack<P>(k < dc ? r[k] : make_uint4(0, 0, 0, 0), f);
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
                const float df = f[e] - Q.q[t][e];
                s = fmaf(df, df, s);
            }
        }
        return group_sum<G>(s);
    }
};

}  // namespace nsg
