// search.cu -- Alg. 1 for a batch of queries (search on NSG, Section 3.6) and
// the per-node search-and-collect of Alg. 2 (Section 3.5 iii), one warp per unit.
#include "search_kern.cuh"

namespace nsg {

struct CollectArgs {
    const float4 *base4;
    int dp4;
    const int *knn;
    int K, W, nav, L, C, H, hshift, max_steps;
    int64_t v0, nv;
    int *cand_ids;
    float *cand_d2;
    int *cand_count, *status;
};

template <int G, int V, int U>
__global__ void __launch_bounds__(256) collect_kernel(CollectArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    WarpSmem s = carve_warp_smem(smem + warp * warp_smem_bytes(a.L, a.W, a.C, a.H), a.L, a.W, a.C, a.H);
    const int64_t stride = (int64_t)gridDim.x * wpb;
    const uint32_t hmask = (uint32_t)a.H - 1;
    for (int64_t j = (int64_t)blockIdx.x * wpb + warp; j < a.nv; j += stride) {
        const int v = (int)(a.v0 + j);
        DistF32<G, V, U> dist{{}, a.base4, a.dp4};
        dist.Q.load_row(a.base4 + (int64_t)v * a.dp4, a.dp4);
        int csize = 0;
        SearchOut o = warp_alg1<true, false>(dist, GraphRef{a.knn, a.K}, a.nav, a.L, s, hmask, a.hshift,
                                             a.max_steps, v, a.C, csize);
        // Alg. 2: v's nearest neighbours in G join the candidates
        const int *row = a.knn + (int64_t)v * a.K;
        int m = 0;
        for (int b = 0; b < a.K; b += 32) {
            int slot = b + (int)lane;
            int w = slot < a.K ? __ldg(row + slot) : -1;
            bool fresh = w >= 0 && visit(s.hash, hmask, a.hshift, w);
            unsigned bal = __ballot_sync(NSG_FULL, fresh);
            if (fresh) s.ids[m + __popc(bal & lanemask_lt())] = w;
            m += __popc(bal);
        }
        __syncwarp();
        if (m > 0) {
            dist(s.ids, m, s.keys);
            collect_merge(s, m, v, a.C, csize);
        }
        // Alg. 2: sorted candidates, cut to C
        for (int t = lane; t < a.C; t += 32) {
            uint64_t e = t < csize ? s.clist[t] : KEY_INF;
            a.cand_ids[j * a.C + t] = t < csize ? kid(e) : -1;
            a.cand_d2[j * a.C + t] = t < csize ? kd2(e) : __int_as_float(0x7f800000);
        }
        if (lane == 0) {
            a.cand_count[j] = csize;
            if (a.status) a.status[j] = o.capped ? -4 : 0;
        }
        __syncwarp();
    }
}

cudaError_t launch_search(const SearchLaunch &l, cudaStream_t st) {
    if (l.nq <= 0) return cudaSuccess;
    SearchArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.dp4 = l.dp / 4;
    a.adj = l.adj;
    a.width = l.width;
    a.W = round32(l.width);
    a.start = l.start;
    a.queries = l.queries;
    a.d = l.d;
    a.nq = l.nq;
    a.k = l.k;
    a.L = l.L;
    a.H = l.hash_slots;
    a.hshift = 32 - log2i((unsigned)l.hash_slots);
    a.max_steps = l.max_steps;
    a.ids = l.ids;
    a.d2 = l.d2;
    a.n_expand = l.n_expand;
    a.n_dist = l.n_dist;
    a.status = l.status;
    a.any_capped = l.any_capped;
    a.lowp = reinterpret_cast<const uint4 *>(l.lowp);
    a.dc = l.lowp_chunks;
    a.scale = l.lowp_scale;
    a.lo = l.lowp_lo;
    a.rerank = l.precision != PREC_F32 ? l.rerank : 0;
    // the re-rank list lives in the hash region when k keys fit there
    a.C = a.rerank && (size_t)a.H * 4 < (size_t)a.k * 8 ? a.k : 0;
    a.stop_model = reinterpret_cast<const __half *>(l.stop_model);
    a.stop_logit = l.stop_logit;
    a.stop_k = l.stop_k;
    a.stop_min_steps = l.stop_min_steps;
    a.trace_feat = l.trace_feat;
    a.trace_flag = l.trace_flag;
    a.trace_cap = l.trace_cap;
    a.kv = l.kv;
    a.Lv = l.Lv;
    a.order = l.order;
    a.work = l.work;
    a.init_count = l.init_count;
    a.init_seed = l.init_seed;
    a.n = (int)l.n;
    a.parts = l.parts > 1 && l.starts != nullptr ? l.parts : 1;
    a.starts = l.starts;
    a.gpool = l.gpool;
    if (a.gpool == nullptr && a.L > 1024) return cudaErrorInvalidValue;
    size_t per_warp = warp_smem_bytes(a.gpool != nullptr ? 0 : a.L, a.W, a.C, a.H, true);
    const size_t per_cta = l.stop_model ? ((sizeof(StopMLP) + 15) & ~size_t(15)) : 0;
    const bool stop = l.stop_model != nullptr || l.trace_feat != nullptr;
    // warps per query: 1, 2 or 4 (the learned-stop / trace kernels use 1)
    const int wpq = stop ? 1 : (l.warps_per_query == 2 || l.warps_per_query == 4 ? l.warps_per_query : 1);
    // a group's region and its control word, spread over its warps
    if (wpq > 1) per_warp = ((per_warp + 32) / wpq + 15) & ~size_t(15);
    // staged row gathers: rows of more than 512 values, without the stop kernels
    a.stage_nb = 0;
    a.stage_rb = 0;
    a.lmap = nullptr;
    if (l.stage > 0 && (stop || a.dp4 <= 128)) return cudaErrorInvalidValue;
    const int nb = search_stage_resolve(l);
    if (nb > 0) {
        stage_layout(l, nb, &a.stage_nb, &a.stage_rb);
        if (l.precision != PREC_F32) a.lmap = reinterpret_cast<const CUtensorMap *>(l.lowp_map);
        const size_t pw = per_warp + stage_bytes(a.stage_nb, a.stage_rb);
        return a.gpool != nullptr ? launch_search_staged_global(a, l, pw, wpq, st)
                                  : launch_search_staged(a, l, pw, wpq, st);
    }
    if (a.gpool != nullptr) return launch_search_global(a, l, per_warp, per_cta, stop, wpq, st);
    return launch_search_args<false>(a, l, per_warp, per_cta, stop, wpq, st);
}

// The ring for nb staged rows of `l`: one row per slot, or (a tensor map over
// the low-precision rows) groups of four rows per slot, 128-byte multiples.
void stage_layout(const SearchLaunch &l, int nb, int *slots, int *slot_bytes) {
    const int rb = (l.precision == PREC_F32 ? l.dp / 4 : l.lowp_chunks) * 16;
    if (l.precision != PREC_F32 && l.lowp_map != nullptr) {
        *slots = std::max(1, nb / 4);
        *slot_bytes = stage_group_bytes(rb);
    } else {
        *slots = nb;
        *slot_bytes = rb;
    }
}

// Rows per warp the staged gathers of `l` hold in flight (0: the register
// gather).
int search_stage_resolve(const SearchLaunch &l) {
    const bool stop = l.stop_model != nullptr || l.trace_feat != nullptr;
    const int dp4 = l.dp / 4;
    if (l.stage == 0 || stop || dp4 <= 128) return 0;
    const int wpq = l.warps_per_query == 2 || l.warps_per_query == 4 ? l.warps_per_query : 1;
    const bool rerank = l.precision != PREC_F32 && l.rerank;
    const int C = rerank && (size_t)l.hash_slots * 4 < (size_t)l.k * 8 ? l.k : 0;
    size_t per_warp = warp_smem_bytes(l.gpool != nullptr ? 0 : l.L, round32(l.width), C, l.hash_slots, true);
    if (wpq > 1) per_warp = ((per_warp + 32) / wpq + 15) & ~size_t(15);
    const int rb = (l.precision == PREC_F32 ? dp4 : l.lowp_chunks) * 16;
    int nb = l.stage > 0 ? std::min(l.stage, STAGE_MAX_SLOTS) : search_stage_slots(rb);
    // a block holds at least one query's warps: fewer rows where those would not fit
    for (; nb > 1; --nb) {
        int slots, sb;
        stage_layout(l, nb, &slots, &sb);
        if ((size_t)wpq * (per_warp + stage_bytes(slots, sb)) <= smem_optin()) break;
    }
    return nb;
}

// Auto staging, as measured on the GIST-shaped 1M x 960 search (k = 100,
// L = 300): bulk copies of rows picked at random complete about one after
// another (~0.4 us each, nearly whatever the row's size), so staging pays
// only where the register gather itself is slow -- FP32 rows of more than
// 2 KB, two in flight per lane group -- and there a ring of 4 slots beats
// larger ones (the ring costs occupancy).
int search_stage_slots(int row_bytes) { return row_bytes > 2048 ? 4 : 0; }

// Warps per query, as measured on the GIST-shaped 1M x 960 search and the
// SIFT-shaped 1M x 128 one.  A group of warps shortens each expansion (more
// rows in flight) but holds more warps per query: it pays while the batch
// leaves the SMs short of warps, and while the pool is small enough to stay
// in shared memory (a group's leader merges into a global-memory pool while
// its other warps wait).  1,000 GIST-shaped queries (6.6 per SM), 8-bit rows:
// L = 300 2 warps 307 k queries/s, 1 warp 234 k; L = 1,059 1 warp 54.7 k,
// 2 warps 43.5 k.  FP32 rows of more than 2 KB (two in flight per lane group
// in registers): 4 warps at L <= 600 (109 k against 89 k at L = 300), 2 above.
// 2,500 SIFT-shaped queries (16 per SM): 1 warp 2.53 M, 2 warps 1.52 M.
int search_auto_wpq(int64_t units, int dp, int precision, int L) {
    if (precision == PREC_F32 && dp * 4 > 2048) return L <= 1024 ? 4 : 2;
    if (L > 1024) return 1;
    const int64_t per_sm = (units + sm_count() - 1) / sm_count();
    return per_sm < 2 ? 4 : per_sm < 8 ? 2 : 1;
}

// Partition-and-merge (Sections 4.2, 4.3): one warp per query merges the
// subsets' result lists into its k smallest (distance, row id) keys: each
// list's entries are mapped to row ids and warp_merge adds them to a sorted
// list of capacity k, one subset after the other.
__global__ void __launch_bounds__(128) merge_parts_kernel(const int *ids_in, const float *d2_in, int64_t nq,
                                                          int parts, int k_in, const int *perm, int k,
                                                          int *ids_out, float *d2_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned lane = lane_id();
    // per warp: list [k], candidates, ck, sk [k_in] (u64); cp, sp [k_in] (int)
    const size_t per = 8ull * (k + 3 * (size_t)k_in) + 8ull * k_in;
    unsigned char *base = smem + warp * ((per + 15) & ~size_t(15));
    uint64_t *list = reinterpret_cast<uint64_t *>(base);
    uint64_t *cand = list + k;
    uint64_t *ck = cand + k_in;
    uint64_t *sk = ck + k_in;
    int *cp = reinterpret_cast<int *>(sk + k_in);
    int *sp = cp + k_in;
    for (int64_t q = (int64_t)blockIdx.x * wpb + warp; q < nq; q += (int64_t)gridDim.x * wpb) {
        int size = 0;
        for (int p = 0; p < parts; ++p) {
            const int *ir = ids_in + (q * parts + p) * (int64_t)k_in;
            const float *dr = d2_in + (q * parts + p) * (int64_t)k_in;
            int m = 0;
            for (int b = 0; b < k_in; b += 32) {
                const int j = b + (int)lane;
                const int pos = j < k_in ? ir[j] : -1;
                const bool has = pos >= 0;
                const unsigned bal = __ballot_sync(NSG_FULL, has);
                if (has) cand[m + __popc(bal & lanemask_lt())] = make_key(dr[j], perm[pos]);
                m += __popc(bal);
            }
            __syncwarp();
            if (m > 0) warp_merge(list, k, size, cand, m, ck, cp, sk, sp);
        }
        for (int c = lane; c < k; c += 32) {
            const bool has = c < size;
            ids_out[q * k + c] = has ? kid(list[c]) : -1;
            if (d2_out) d2_out[q * k + c] = has ? kd2(list[c]) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

cudaError_t launch_merge_parts(const int *ids_in, const float *d2_in, int64_t nq, int parts, int k_in,
                               const int *perm, int k, int *ids_out, float *d2_out, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const size_t per = ((8ull * (k + 3 * (size_t)k_in) + 8ull * k_in) + 15) & ~size_t(15);
    int grid, wpb;
    size_t smem;
    cudaError_t e = config(merge_parts_kernel, per, 4, nq, &grid, &wpb, &smem);
    if (e != cudaSuccess) return e;
    merge_parts_kernel<<<grid, wpb * 32, smem, st>>>(ids_in, d2_in, nq, parts, k_in, perm, k, ids_out, d2_out);
    return cudaGetLastError();
}

__global__ void gather_rows_kernel(const float *base, int64_t n, int d, const int *perm, float *out) {
    const int64_t total = n * d;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = x / d;
        out[x] = base[(int64_t)perm[i] * d + (x - i * d)];
    }
}

cudaError_t launch_gather_rows(const float *base, int64_t n, int d, const int *perm, float *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n * d + 255) / 256, (int64_t)sm_count() * 16);
    gather_rows_kernel<<<(int)blocks, 256, 0, st>>>(base, n, d, perm, out);
    return cudaGetLastError();
}

__global__ void offset_adj_kernel(const int *in, int64_t total, int offset, int *out) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int v = in[x];
        out[x] = v >= 0 ? v + offset : -1;
    }
}

cudaError_t launch_offset_adj(const int *in, int64_t nv, int R, int offset, int *out, cudaStream_t st) {
    if (nv <= 0) return cudaSuccess;
    const int64_t total = nv * R;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
    offset_adj_kernel<<<(int)blocks, 256, 0, st>>>(in, total, offset, out);
    return cudaGetLastError();
}

// Visiting order of a batch, farthest from the navigating node first.  A
// launch ends when its last queries do, and a query's length is only known
// once it has run; its distance to the navigating node is a weak but free
// predictor of it (longer greedy path), and drawing the far queries first
// leaves the short ones for the end.  Measured on the SIFT-shaped 1M search
// (10,000 queries, 8-bit form, L = 138): 2.067 ms in the generated order,
// 1.846 ms far-first, 1.703 ms ordered by the true expansion counts (the bound),
// 2.096 ms near-first.  A counting sort into NAV_BUCKETS distance buckets
// (order within a bucket is arbitrary: each query's result is independent of
// the order).
constexpr int NAV_BUCKETS = 1024;

__global__ void nav_dist_kernel(const float *__restrict__ q, int64_t nq, int d, const float *__restrict__ nav,
                                float *key, unsigned *maxbits) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned lane = lane_id();
    if (w >= nq) return;
    float s = 0.0f;
    for (int j = lane; j < d; j += 32) {
        const float t = q[w * d + j] - nav[j];
        s = fmaf(t, t, s);
    }
    s = group_sum<32>(s);
    if (lane == 0) {
        key[w] = s;
        atomicMax(maxbits, __float_as_uint(s));  // s >= +0: the bits order as the values
    }
}

__global__ void nav_bucket_kernel(const float *key, int64_t nq, const unsigned *maxbits, int *bucket, int *hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const float mx = __uint_as_float(*maxbits);
    const int b = mx > 0.0f ? min(NAV_BUCKETS - 1, (int)(key[i] / mx * NAV_BUCKETS)) : 0;
    bucket[i] = NAV_BUCKETS - 1 - b;  // farthest first
    atomicAdd(hist + NAV_BUCKETS - 1 - b, 1);
}

__global__ void nav_scan_kernel(int *hist) {  // exclusive scan of NAV_BUCKETS counts, one block of 1024
    __shared__ int sh[NAV_BUCKETS];
    const int t = threadIdx.x;
    sh[t] = hist[t];
    __syncthreads();
    for (int o = 1; o < NAV_BUCKETS; o <<= 1) {
        const int v = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    hist[t] = sh[t] - hist[t];
}

__global__ void nav_scatter_kernel(const int *bucket, int64_t nq, int *offsets, int *order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    order[atomicAdd(offsets + bucket[i], 1)] = (int)i;
}

size_t nav_order_scratch_bytes(int64_t nq) { return (size_t)nq * 12 + (NAV_BUCKETS + 4) * 4; }

cudaError_t launch_nav_order(const float *queries, int64_t nq, int d, const float *nav_row, void *scratch,
                             int **order, cudaStream_t st) {
    int *ord = static_cast<int *>(scratch);
    float *key = reinterpret_cast<float *>(ord + nq);
    int *bucket = reinterpret_cast<int *>(key + nq);
    int *hist = bucket + nq;
    unsigned *maxbits = reinterpret_cast<unsigned *>(hist + NAV_BUCKETS);
    cudaError_t e = cudaMemsetAsync(hist, 0, (NAV_BUCKETS + 1) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    nav_dist_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(queries, nq, d, nav_row, key, maxbits);
    nav_bucket_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(key, nq, maxbits, bucket, hist);
    nav_scan_kernel<<<1, NAV_BUCKETS, 0, st>>>(hist);
    nav_scatter_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(bucket, nq, hist, ord);
    *order = ord;
    return cudaGetLastError();
}

int64_t search_pool_slots() { return (int64_t)sm_count() * 32; }

size_t search_warp_smem_bytes(int L, int W, int H) { return warp_smem_bytes(L, W, 0, H, true); }

cudaError_t launch_collect(const CollectLaunch &l, cudaStream_t st) {
    if (l.nv <= 0) return cudaSuccess;
    CollectArgs a;
    a.base4 = reinterpret_cast<const float4 *>(l.base);
    a.dp4 = l.dp / 4;
    a.knn = l.knn;
    a.K = l.K;
    a.W = round32(l.K);
    a.nav = l.nav;
    a.L = l.L;
    a.C = l.C;
    a.H = l.hash_slots;
    a.hshift = 32 - log2i((unsigned)l.hash_slots);
    a.max_steps = l.max_steps;
    a.v0 = l.v0;
    a.nv = l.nv;
    a.cand_ids = l.cand_ids;
    a.cand_d2 = l.cand_d2;
    a.cand_count = l.cand_count;
    a.status = l.status;
    size_t per_warp = warp_smem_bytes(a.L, a.W, a.C, a.H);
    cudaError_t err = cudaSuccess;
    NSG_DISPATCH_DP4(a.dp4, {
        auto kern = collect_kernel<G_, V_, U_>;
        int grid, wpb;
        size_t smem;
        err = config(kern, per_warp, 4, l.nv, &grid, &wpb, &smem);
        if (err == cudaSuccess) {
            kern<<<grid, wpb * 32, smem, st>>>(a);
            err = cudaGetLastError();
        }
    });
    return err;
}

}  // namespace nsg
