// capi.cu -- the extern "C" entry points declared in include/nsg.h.
//
// Host code here only validates arguments, owns index memory and sequences
// launches; every step of the method runs in the kernels of search.cu,
// build.cu and knn.cu.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <vector>

#include "kernels.h"
#include "nsg.h"

constexpr unsigned kWorkSlots = 256;

struct nsg_index {
    int64_t n = 0;
    int d = 0, dp = 0, R = 0, nav = 0;
    float *base = nullptr;  // [n][dp], zero padded
    int *adj = nullptr;     // [n][R], -1 padded
    int *deg = nullptr;     // [n]
    int *flag = nullptr;    // [4] device scratch for nsg_search's cap check
    // work counters of the search launches (warps draw queries from one),
    // used round-robin so concurrent calls on other streams take other slots
    int *work = nullptr;    // [kWorkSlots]
    mutable std::atomic<unsigned> work_next{0};
    // low-precision copies, indexed by nsg_precision (1 = BF16, 2 = FP8-e4m3, 3 = U8)
    void *lowp[4] = {nullptr, nullptr, nullptr, nullptr};  // by nsg_precision
    int lowp_dpl[4] = {0, 0, 0, 0};         // values per row (16-byte multiple)
    float lowp_scale[4] = {1, 1, 1, 1};     // query multiplier
    float lowp_lo[4] = {0, 0, 0, 0};        // U8 offset
    int lowp_exact[4] = {0, 0, 0, 0};       // every value (U8: every distance) survived
    void *lowp_map[4] = {nullptr, nullptr, nullptr, nullptr};  // device tensor maps for staged four-row gathers
    int max_degree = 0;
    double avg_degree = 0.0;
    int64_t n_fixup = 0;
    int64_t n_fixup_searches = 0;  // fix-ups whose speculative search was stale and ran again
    int64_t prune_examined = 0;    // candidates the edge selection examined, all nodes
    int knn_iters = 0;             // nn-descent iterations of the kNN stage (0: exact kNN)
    float ms[6] = {0, 0, 0, 0, 0, 0};
    // nsg_search_host: device staging for `host_cap` queries of up to
    // `host_k` results and a step-cap flag; one call at a time
    mutable std::mutex host_mu;
    mutable int64_t host_cap = 0;
    mutable int host_k = 0;
    mutable float *host_q = nullptr;
    mutable int *host_ids = nullptr;
    mutable float *host_d2 = nullptr;
    mutable int *host_flag = nullptr;
    // partitioned index (Sections 4.2, 4.3): the subsets' graphs side by side,
    // subset p at positions [part_off[p], part_off[p+1]); starts [parts] device
    // (each subset's navigating node), perm [n] device (position -> row id)
    int parts = 1;
    int *starts = nullptr;
    int *perm = nullptr;
    std::vector<int64_t> part_off;
    // nsg_search_partitioned: per-unit results before the merge, grown on demand
    mutable std::mutex part_mu;
    mutable int64_t part_cap = 0;
    mutable int *part_ids = nullptr;
    mutable float *part_d2 = nullptr;
    // global-memory search pools (nsg_search_params.pool): one slot of L keys
    // per resident warp, grown on demand
    mutable std::mutex gpool_mu;
    mutable uint64_t *gpool = nullptr;
    mutable size_t gpool_bytes = 0;
};

namespace {

thread_local char g_err[512] = "";
// kNN engine: tensor cores when the answer is exact, else the CUDA-core scan;
// NSG_KNN_ENGINE=scan forces the CUDA-core scan (read at every call).
bool knn_force_scan() {
    const char *e = std::getenv("NSG_KNN_ENGINE");
    return e && std::strcmp(e, "scan") == 0;
}

nsg_status cuda_fail(cudaError_t e, const char *what) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return NSG_ECUDA;
}

// Runs f() and turns a failed host allocation into NSG_ENOMEM, so that no
// exception leaves the C ABI.
template <class F>
nsg_status host_guard(F &&f) {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return NSG_ENOMEM;
    } catch (const std::length_error &) {
        return NSG_ENOMEM;
    }
}

#define NSG_CK(x)                                                \
    do {                                                         \
        cudaError_t e_ = (x);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x);         \
    } while (0)

// RAII device buffer for scratch and index members under construction.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t count) {
        if (p) cudaFree(p);
        p = nullptr;
        return cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    }
    T *release() {
        T *q = p;
        p = nullptr;
        return q;
    }
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
inline int round_up4(int d) { return (d + 3) & ~3; }
inline unsigned next_pow2(unsigned x) {
    unsigned p = 1;
    while (p < x) p <<= 1;
    return p;
}
// Visited-set slots per query of the build's searches (collect, connectivity).
// Small on purpose: the set may forget (results do not change), and 2 KB per
// warp keeps the build kernels' occupancy.
inline int default_hash(int L, int width) {
    (void)width;
    return L <= 1024 ? 512 : 2048;  // longer searches measure more nodes
}

// Visited-set slots per query of nsg_search / nsg_search_ex: 1024 when the
// searches still hold 32 warps per SM with it (the search kernels keep the
// merge's sorted keys in the candidate keys' space), else 512.  Measured on
// the SIFT-shaped 1M at L = 138 (10,000 queries): 1024 slots re-measure 9 %
// fewer nodes and run 2-3 % faster than 512 in every form; where 1024 slots
// cost resident warps (L = 150 and up at R = 50) they are slower.
// Visited-set slots of a search when the caller leaves them to the library.
// A forgotten id is measured again (same key, same results), so a larger set
// saves distances and costs shared memory: a batch that leaves the SMs short
// of warps (units search regions, wpq warps each, fewer than 32 warps per SM)
// takes the largest set up to 4,096 slots whose regions still fit one wave
// (GIST-shaped 1M, 1,000 queries, 8-bit, 2 warps per query, L = 300: 14,260
// distances per query and 303 k queries/s with 512 slots, 9,518 and 355 k with
// 4,096; 8,192 no longer fit one wave: 251 k); pools above 1024 keys (in
// global memory) up to 8,192 slots.  Searches whose rows go through a staging
// ring, and full batches: 2048 above L = 1024, else 1024 when the search
// still holds 32 warps per SM with it, else 512.
inline int default_search_hash(int L, int width, int64_t units = 0, int wpq = 1, bool staged = false) {
    static int smem_sm = 0, reserved = 0;
    if (!smem_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    }
    const int W = (width + 31) & ~31;
    const int64_t sms = nsg::sm_count();
    const int64_t regions = (units + sms - 1) / sms;  // per SM, one wave
    const int Ls = L > 1024 ? 0 : L;                  // pools above 1024 keys live in global memory
    if (!staged && units > 0 && regions * wpq < 32 && smem_sm > 0) {
        const int rpb = wpq < 4 ? 4 / wpq : 1;  // regions per block of 4 warps
        const int64_t blocks = (regions + rpb - 1) / rpb;
        for (int H = L > 1024 ? 8192 : 4096; H >= (L > 1024 ? 2048 : 1024); H >>= 1) {
            const size_t region = nsg::search_warp_smem_bytes(Ls, W, H) + 32;
            if (blocks * (rpb * region + (size_t)reserved) <= (size_t)smem_sm) return H;
        }
    }
    if (L > 1024) return 2048;
    const size_t per_block = 4 * nsg::search_warp_smem_bytes(L, W, 1024) + (size_t)reserved;
    return smem_sm > 0 && 8 * per_block <= (size_t)smem_sm ? 1024 : 512;
}
inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Published SplitMix64 finaliser (Steele, Lea, Flood 2014): the random start
// node of Alg. 2 is splitmix64(seed) mod n.
inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void check_ids_kernel(const int *ids, int64_t count, int64_t n, int *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < count;
         x += (int64_t)gridDim.x * blockDim.x) {
        int v = ids[x];
        if (v < -1 || v >= n) atomicOr(bad, 1);
    }
}

// Every id in [-1, n)?  Guards the gather kernels against out-of-range reads.
nsg_status check_ids(const int *ids, int64_t count, int64_t n, cudaStream_t st) {
    if (count <= 0) return NSG_OK;
    DevBuf<int> bad;
    NSG_CK(bad.alloc(1));
    NSG_CK(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    int64_t blocks = (count + 255) / 256;
    int64_t cap = (int64_t)nsg::sm_count() * 8;
    check_ids_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, st>>>(ids, count, n, bad.p);
    NSG_CK(cudaGetLastError());
    int h = 0;
    NSG_CK(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    return h ? NSG_EINVAL : NSG_OK;
}

// Copy [n][d] into a fresh zero-padded [n][dp] buffer.
nsg_status padded_copy(const float *src, int64_t n, int d, int dp, DevBuf<float> &dst, cudaStream_t st) {
    NSG_CK(dst.alloc((size_t)n * dp));
    NSG_CK(nsg::launch_pad_rows(src, n, d, dst.p, dp, st));
    return NSG_OK;
}

// Returns a [n][dp] view: the input itself when already padded and aligned.
nsg_status padded_view(const float *src, int64_t n, int d, DevBuf<float> &tmp, const float **view,
                       cudaStream_t st) {
    if ((d & 3) == 0 && aligned16(src)) {
        *view = src;
        return NSG_OK;
    }
    nsg_status s = padded_copy(src, n, d, round_up4(d), tmp, st);
    *view = tmp.p;
    return s;
}

nsg_status knn_run(const float *bp, int64_t n, int dp, const float *qp, int64_t nq, int64_t q0, int k,
                   int self_join, int *ids, float *d2, cudaStream_t st) {
    nsg::KnnLaunch l;
    l.base = bp;
    l.n = n;
    l.dp = dp;
    l.queries = qp;
    l.nq = nq;
    l.q0 = q0;
    l.k = k;
    l.self_join = self_join;
    l.ids = ids;
    l.d2 = d2;
    int used = 0;
    if (!knn_force_scan()) NSG_CK(nsg::launch_knn_tc(l, &used, st));
    if (!used) NSG_CK(nsg::launch_knn_direct(l, st));
    return NSG_OK;
}

bool nndescent_params_ok(const nsg_nndescent_params &p) {
    return p.sample >= 1 && p.sample <= 256 && p.reverse >= 0 && p.reverse <= 256 && p.iters >= 0 &&
           p.iters <= 1000 && p.delta >= 0.0f;
}

// Approximate kNN graph by nn-descent into ids [n][K] (d2 nullable), with
// scratch allocated for the call.  base [n][dp] padded rows of d values.
// Integer data of span <= 255 with d * 255^2 < 2^24 (every distance an exact
// integer below 2^24) get an 8-bit copy x - min for the distances: the same
// keys as the FP32 rows at a quarter of the bytes gathered.
nsg_status nndescent_run(const float *base, int64_t n, int dp, int d, int K, const nsg_nndescent_params &p,
                         int *ids, float *d2, int *iters_run, int64_t *last_updates, cudaStream_t st) {
    DevBuf<unsigned char> scratch, u8;
    NSG_CK(scratch.alloc(nsg::nndescent_scratch_bytes(n, K, p.sample, p.reverse)));
    float lo = 0.0f;
    bool use_u8 = false;
    const int dpl = (d + 15) / 16 * 16;
    if ((int64_t)d * 65025 < (1 << 24)) {
        DevBuf<unsigned> flags;
        NSG_CK(flags.alloc(4));
        unsigned mm[3] = {0xffffffffu, 0u, 0u};
        NSG_CK(cudaMemcpyAsync(flags.p, mm, sizeof(mm), cudaMemcpyHostToDevice, st));
        NSG_CK(nsg::launch_minmax(base, n, dp, d, flags.p, st));
        NSG_CK(cudaMemcpyAsync(mm, flags.p, sizeof(mm), cudaMemcpyDeviceToHost, st));
        NSG_CK(cudaStreamSynchronize(st));
        const float mn = nsg::float_from_order_key(mm[0]), mx = nsg::float_from_order_key(mm[1]);
        if (mm[2] == 0 && (double)mx - (double)mn <= 255.0) {
            lo = mn;
            NSG_CK(cudaMemsetAsync(flags.p, 0, sizeof(unsigned), st));
            NSG_CK(u8.alloc((size_t)n * dpl));
            NSG_CK(nsg::launch_to_lowp(base, n, dp, d, NSG_PREC_U8, 1.0f, lo, u8.p, dpl,
                                       reinterpret_cast<int *>(flags.p), st));
            unsigned inexact = 0;
            NSG_CK(cudaMemcpyAsync(&inexact, flags.p, sizeof(inexact), cudaMemcpyDeviceToHost, st));
            NSG_CK(cudaStreamSynchronize(st));
            use_u8 = inexact == 0;
        }
    }
    nsg::NnDescentLaunch l;
    l.u8 = use_u8 ? u8.p : nullptr;
    l.u8_chunks = dpl / 16;
    l.u8_lo = lo;
    l.d = d;
    l.base = base;
    l.n = n;
    l.dp = dp;
    l.K = K;
    l.S = p.sample;
    l.Sr = p.reverse;
    l.iters = p.iters;
    l.delta = p.delta;
    l.seed = p.seed;
    l.ids = ids;
    l.d2 = d2;
    l.scratch = scratch.p;
    l.iters_run = iters_run;
    l.last_updates = last_updates;
    NSG_CK(nsg::launch_nndescent(l, st));
    NSG_CK(cudaStreamSynchronize(st));
    return NSG_OK;
}

nsg_status navigate_run(const float *base, int64_t n, int d, const int *knn, int K, const double *c,
                        int start, int L, int *nav_host, cudaStream_t st) {
    DevBuf<uint32_t> visited;
    DevBuf<int> out;
    NSG_CK(visited.alloc((size_t)(n + 31) / 32));
    NSG_CK(out.alloc(2));
    NSG_CK(cudaMemsetAsync(visited.p, 0, sizeof(uint32_t) * ((n + 31) / 32), st));
    NSG_CK(nsg::launch_navigate(base, n, d, knn, K, c, start, L, visited.p, nsg::default_steps(L), out.p,
                                out.p + 1, st));
    int h[2] = {0, 0};
    NSG_CK(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    *nav_host = h[0];
    return h[1] ? NSG_ESTEPCAP : NSG_OK;
}

nsg_status connect_run(const float *bp, int64_t n, int dp, int *adj, int *deg, int R, int nav, int L,
                       int *n_added, cudaStream_t st, int *n_research = nullptr) {
    nsg::ConnectLaunch c;
    c.base = bp;
    c.n = n;
    c.dp = dp;
    c.adj = adj;
    c.deg = deg;
    c.R = R;
    c.nav = nav;
    c.L = L;
    c.hash_slots = default_hash(L, R);
    c.max_steps = nsg::default_steps(L);
    int h[4] = {0, 0, 0, 0};
    NSG_CK(nsg::run_connect(c, h, st));
    if (n_added) *n_added = h[0];
    if (n_research) *n_research = h[3];
    if (h[1] == NSG_EDEGREE) return NSG_EDEGREE;
    return h[2] ? NSG_ESTEPCAP : NSG_OK;
}

nsg_status collect_prune_all(const float *bp, int64_t n, int dp, const int *knn, int K, int nav, int L,
                             int R, int C, int *adj, int *deg, float *ms_collect, float *ms_prune,
                             int64_t *examined, cudaStream_t st) {
    // candidate lists are materialised for a chunk of nodes at a time
    const size_t budget = size_t(2) << 30;
    int64_t chunk = (int64_t)(budget / ((size_t)C * 8 + 8));
    if (chunk > n) chunk = n;
    if (chunk < 1) chunk = 1;
    DevBuf<int> cid, ccnt;
    DevBuf<float> cd2;
    DevBuf<unsigned long long> nexam;
    NSG_CK(cid.alloc((size_t)chunk * C));
    NSG_CK(cd2.alloc((size_t)chunk * C));
    NSG_CK(ccnt.alloc(chunk));
    NSG_CK(nexam.alloc(1));
    NSG_CK(cudaMemsetAsync(nexam.p, 0, sizeof(unsigned long long), st));
    cudaEvent_t ev[3];
    for (auto &e : ev) NSG_CK(cudaEventCreate(&e));
    float tc = 0, tp = 0;
    nsg_status rc = NSG_OK;
    for (int64_t v0 = 0; v0 < n && rc == NSG_OK; v0 += chunk) {
        int64_t nv = n - v0 < chunk ? n - v0 : chunk;
        nsg::CollectLaunch c;
        c.base = bp;
        c.n = n;
        c.dp = dp;
        c.knn = knn;
        c.K = K;
        c.nav = nav;
        c.L = L;
        c.C = C;
        c.v0 = v0;
        c.nv = nv;
        c.hash_slots = default_hash(L, K);
        c.max_steps = nsg::default_steps(L);
        c.cand_ids = cid.p;
        c.cand_d2 = cd2.p;
        c.cand_count = ccnt.p;
        c.status = nullptr;
        cudaEventRecord(ev[0], st);
        cudaError_t e = nsg::launch_collect(c, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "launch_collect");
        cudaEventRecord(ev[1], st);
        nsg::PruneLaunch p;
        p.base = bp;
        p.n = n;
        p.dp = dp;
        p.cand_ids = cid.p;
        p.cand_d2 = cd2.p;
        p.cand_count = ccnt.p;
        p.C = C;
        p.R = R;
        p.v0 = v0;
        p.nv = nv;
        p.adj = adj;
        p.deg = deg;
        p.examined = nexam.p;
        if (rc == NSG_OK) {
            e = nsg::launch_prune(p, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "launch_prune");
        }
        cudaEventRecord(ev[2], st);
        e = cudaEventSynchronize(ev[2]);
        if (e != cudaSuccess && rc == NSG_OK) rc = cuda_fail(e, "collect/prune");
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        tc += a;
        tp += b;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (ms_collect) *ms_collect = tc;
    if (ms_prune) *ms_prune = tp;
    if (examined && rc == NSG_OK) {
        unsigned long long h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, nexam.p, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "prune counter");
        *examined = (int64_t)h;
    }
    return rc;
}

nsg_status finish_index_body(nsg_index *ix, cudaStream_t st) {
    std::vector<int> deg((size_t)ix->n);
    NSG_CK(cudaMemcpyAsync(deg.data(), ix->deg, sizeof(int) * ix->n, cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    int64_t sum = 0;
    int mx = 0;
    for (int v : deg) {
        sum += v;
        mx = v > mx ? v : mx;
    }
    ix->max_degree = mx;
    ix->avg_degree = ix->n ? (double)sum / (double)ix->n : 0.0;
    NSG_CK(cudaMalloc(reinterpret_cast<void **>(&ix->flag), 4 * sizeof(int)));
    NSG_CK(cudaMalloc(reinterpret_cast<void **>(&ix->work), kWorkSlots * sizeof(int)));
    return NSG_OK;
}

nsg_status finish_index(nsg_index *ix, cudaStream_t st) {
    return host_guard([&] { return finish_index_body(ix, st); });
}

void destroy(nsg_index *ix) {
    if (!ix) return;
    if (ix->base) cudaFree(ix->base);
    if (ix->adj) cudaFree(ix->adj);
    if (ix->deg) cudaFree(ix->deg);
    if (ix->flag) cudaFree(ix->flag);
    if (ix->work) cudaFree(ix->work);
    for (void *p : ix->lowp)
        if (p) cudaFree(p);
    for (void *p : ix->lowp_map)
        if (p) cudaFree(p);
    if (ix->host_q) cudaFree(ix->host_q);
    if (ix->host_ids) cudaFree(ix->host_ids);
    if (ix->host_d2) cudaFree(ix->host_d2);
    if (ix->host_flag) cudaFree(ix->host_flag);
    if (ix->starts) cudaFree(ix->starts);
    if (ix->perm) cudaFree(ix->perm);
    if (ix->part_ids) cudaFree(ix->part_ids);
    if (ix->part_d2) cudaFree(ix->part_d2);
    if (ix->gpool) cudaFree(ix->gpool);
    delete ix;
}

double since_ms(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

namespace nsg {

void record_cuda_error(cudaError_t e, const char *what) { cuda_fail(e, what); }

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev] > 0 ? cache[dev] : 1;
}

size_t smem_optin() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return cache[dev] > 0 ? (size_t)cache[dev] : 48 * 1024;
}

size_t smem_per_sm() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    return cache[dev] > 0 ? (size_t)cache[dev] : 64 * 1024;
}

}  // namespace nsg

extern "C" {

const char *nsg_status_str(nsg_status s) {
    switch (s) {
    case NSG_OK: return "NSG_OK";
    case NSG_EINVAL: return "NSG_EINVAL: invalid argument";
    case NSG_ENOMEM: return "NSG_ENOMEM: allocation failed";
    case NSG_ECUDA: return "NSG_ECUDA: CUDA runtime error";
    case NSG_ESTEPCAP: return "NSG_ESTEPCAP: a search hit its step cap";
    case NSG_EDEGREE: return "NSG_EDEGREE: no reached node has a free adjacency slot";
    case NSG_EIO: return "NSG_EIO: file error";
    case NSG_EFORMAT: return "NSG_EFORMAT: not an NSG index file";
    }
    return "unknown nsg_status";
}

const char *nsg_last_cuda_error(void) { return g_err; }

nsg_status nsg_knn_init(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t *knn_ids_dev,
                        float *knn_d2_dev, void *stream) {
    if (!base_dev || !knn_ids_dev || n < 2 || d < 1 || d > 4 * nsg::MAX_DP4_HOST || K < 1 || K >= n ||
        K > 256 || n >= INT32_MAX)
        return NSG_EINVAL;
    cudaStream_t st = S(stream);
    DevBuf<float> tmp;
    const float *bp = nullptr;
    nsg_status s = padded_view(base_dev, n, d, tmp, &bp, st);
    if (s) return s;
    return knn_run(bp, n, round_up4(d), bp, n, 0, K, 1, knn_ids_dev, knn_d2_dev, st);
}

nsg_status nsg_knn_query(const float *base_dev, int64_t n, int32_t d, const float *queries_dev,
                         int64_t nq, int32_t k, int32_t *ids_dev, float *d2_dev, void *stream) {
    if (!base_dev || n < 1 || d < 1 || d > 4 * nsg::MAX_DP4_HOST || k < 1 || k > 256 || k > n ||
        nq < 0 || n >= INT32_MAX)
        return NSG_EINVAL;
    if (nq == 0) return NSG_OK;
    if (!queries_dev || !ids_dev) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    DevBuf<float> tb, tq;
    const float *bp = nullptr, *qp = nullptr;
    nsg_status s = padded_view(base_dev, n, d, tb, &bp, st);
    if (!s) s = padded_view(queries_dev, nq, d, tq, &qp, st);
    if (s) return s;
    return knn_run(bp, n, round_up4(d), qp, nq, 0, k, 0, ids_dev, d2_dev, st);
}

nsg_status nsg_centroid(const float *base_dev, int64_t n, int32_t d, double *centroid_dev, void *stream) {
    if (!base_dev || !centroid_dev || n < 1 || d < 1) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    int nb = nsg::sm_count() * 4;
    DevBuf<double> part;
    NSG_CK(part.alloc((size_t)nb * d));
    NSG_CK(nsg::launch_centroid(base_dev, n, d, part.p, nb, centroid_dev, st));
    NSG_CK(cudaStreamSynchronize(st));  // scratch is freed on return
    return NSG_OK;
}

nsg_status nsg_navigate(const float *base_dev, int64_t n, int32_t d, const int32_t *knn_ids_dev,
                        int32_t K, const double *centroid_dev, int32_t start, int32_t L,
                        int32_t *nav_host, void *stream) {
    if (!base_dev || !knn_ids_dev || !centroid_dev || !nav_host || n < 1 || d < 1 ||
        d > 4 * nsg::MAX_DP4_HOST || K < 1 || L < 1 || L > 1024 || start < 0 || start >= n)
        return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg_status s = check_ids(knn_ids_dev, n * K, n, st);
    if (s) return s;
    return navigate_run(base_dev, n, d, knn_ids_dev, K, centroid_dev, start, L, nav_host, st);
}

nsg_status nsg_collect(const float *base_dev, int64_t n, int32_t d, const int32_t *knn_ids_dev,
                       int32_t K, int32_t nav, int32_t L, int32_t C, int64_t v0, int64_t nv,
                       int32_t *cand_ids_dev, float *cand_d2_dev, int32_t *cand_count_dev,
                       int32_t *status_dev, void *stream) {
    if (!base_dev || !knn_ids_dev || (d & 3) || !aligned16(base_dev) || d < 4 ||
        d > 4 * nsg::MAX_DP4_HOST || n < 1 || K < 1 || K > 1024 || L < 1 || L > 1024 || C < 1 ||
        C > 4096 || nav < 0 || nav >= n || v0 < 0 || nv < 0 || v0 + nv > n)
        return NSG_EINVAL;
    if (nv == 0) return NSG_OK;
    if (!cand_ids_dev || !cand_d2_dev || !cand_count_dev) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg_status s = check_ids(knn_ids_dev, n * K, n, st);
    if (s) return s;
    nsg::CollectLaunch c;
    c.base = base_dev;
    c.n = n;
    c.dp = d;
    c.knn = knn_ids_dev;
    c.K = K;
    c.nav = nav;
    c.L = L;
    c.C = C;
    c.v0 = v0;
    c.nv = nv;
    c.hash_slots = default_hash(L, K);
    c.max_steps = nsg::default_steps(L);
    c.cand_ids = cand_ids_dev;
    c.cand_d2 = cand_d2_dev;
    c.cand_count = cand_count_dev;
    c.status = status_dev;
    NSG_CK(nsg::launch_collect(c, st));
    return NSG_OK;
}

nsg_status nsg_prune(const float *base_dev, int64_t n, int32_t d, const int32_t *cand_ids_dev,
                     const float *cand_d2_dev, const int32_t *cand_count_dev, int32_t C, int32_t R,
                     int64_t v0, int64_t nv, int32_t *adj_dev, int32_t *deg_dev, void *stream) {
    if (!base_dev || (d & 3) || !aligned16(base_dev) || d < 4 || d > 4 * nsg::MAX_DP4_HOST || n < 1 ||
        C < 1 || R < 1 || R > 1024 || v0 < 0 || nv < 0 || v0 + nv > n)
        return NSG_EINVAL;
    if (nv == 0) return NSG_OK;
    if (!cand_ids_dev || !cand_d2_dev || !cand_count_dev || !adj_dev || !deg_dev) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg_status s = check_ids(cand_ids_dev, nv * C, n, st);
    if (s) return s;
    nsg::PruneLaunch p;
    p.base = base_dev;
    p.n = n;
    p.dp = d;
    p.cand_ids = cand_ids_dev;
    p.cand_d2 = cand_d2_dev;
    p.cand_count = cand_count_dev;
    p.C = C;
    p.R = R;
    p.v0 = v0;
    p.nv = nv;
    p.adj = adj_dev;
    p.deg = deg_dev;
    NSG_CK(nsg::launch_prune(p, st));
    return NSG_OK;
}

nsg_status nsg_connect(const float *base_dev, int64_t n, int32_t d, int32_t *adj_dev, int32_t *deg_dev,
                       int32_t R, int32_t nav, int32_t L, int32_t *n_added_host, void *stream) {
    if (!base_dev || !adj_dev || !deg_dev || (d & 3) || !aligned16(base_dev) || d < 4 ||
        d > 4 * nsg::MAX_DP4_HOST || n < 1 || R < 1 || R > 1024 || L < 1 || L > 1024 || nav < 0 ||
        nav >= n)
        return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg_status s = check_ids(adj_dev, n * R, n, st);
    if (s) return s;
    return connect_run(base_dev, n, d, adj_dev, deg_dev, R, nav, L, n_added_host, st);
}

nsg_status nsg_build_naive(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t R, uint64_t seed,
                           void *stream, nsg_index **out) {
    if (!out) return NSG_EINVAL;
    *out = nullptr;
    if (!base_dev || n < 2 || n >= INT32_MAX || d < 1 || d > 4 * nsg::MAX_DP4_HOST || K < 1 || K >= n ||
        K > 256 || R < 1 || R > 1024)
        return NSG_EINVAL;
    cudaStream_t st = S(stream);
    auto t_all = std::chrono::steady_clock::now();
    nsg_index *ix = new (std::nothrow) nsg_index;
    if (!ix) return NSG_ENOMEM;
    ix->n = n;
    ix->d = d;
    ix->dp = round_up4(d);
    ix->R = R;
    DevBuf<float> base, kd;
    DevBuf<int> adj, deg, knn;
    nsg_status s = padded_copy(base_dev, n, d, ix->dp, base, st);
    cudaError_t e = cudaSuccess;
    if (!s && (e = adj.alloc((size_t)n * R)) != cudaSuccess) s = cuda_fail(e, "alloc adj");
    if (!s && (e = deg.alloc((size_t)n)) != cudaSuccess) s = cuda_fail(e, "alloc deg");
    if (!s && (e = knn.alloc((size_t)n * K)) != cudaSuccess) s = cuda_fail(e, "alloc knn");
    if (!s && (e = kd.alloc((size_t)n * K)) != cudaSuccess) s = cuda_fail(e, "alloc knn d2");
    // the kNN graph (ids and distances, in key order per row) ...
    auto t0 = std::chrono::steady_clock::now();
    if (!s) s = knn_run(base.p, n, ix->dp, base.p, n, 0, K, 1, knn.p, kd.p, st);
    if (!s && (e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(e, "knn");
    ix->ms[0] = (float)since_ms(t0);
    // ... whose rows are every node's candidates for the MRNG selection
    t0 = std::chrono::steady_clock::now();
    if (!s) {
        nsg::PruneLaunch p;
        p.base = base.p;
        p.n = n;
        p.dp = ix->dp;
        p.cand_ids = knn.p;
        p.cand_d2 = kd.p;
        p.cand_count = nullptr;
        p.C = K;
        p.R = R;
        p.v0 = 0;
        p.nv = n;
        p.adj = adj.p;
        p.deg = deg.p;
        if ((e = nsg::launch_prune(p, st)) != cudaSuccess) s = cuda_fail(e, "launch_prune");
        if (!s && (e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(e, "prune");
    }
    ix->ms[3] = (float)since_ms(t0);
    ix->nav = (int)(splitmix64(seed) % (uint64_t)n);  // a random start node; no navigating node
    if (s) {
        destroy(ix);
        return s;
    }
    ix->base = base.release();
    ix->adj = adj.release();
    ix->deg = deg.release();
    s = finish_index(ix, st);
    ix->ms[5] = (float)since_ms(t_all);
    if (s) {
        destroy(ix);
        return s;
    }
    *out = ix;
    return NSG_OK;
}

static nsg_status build_index(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                       int32_t C, uint64_t seed, const nsg_nndescent_params *nnd, void *stream, nsg_index **out) {
    if (!out) return NSG_EINVAL;
    *out = nullptr;
    if (!base_dev || n < 2 || n >= INT32_MAX || d < 1 || d > 4 * nsg::MAX_DP4_HOST || K < 1 || K >= n ||
        K > 256 || L < 1 || L > 1024 || R < 1 || R > 1024 || C < R || C > 4096)
        return NSG_EINVAL;
    cudaStream_t st = S(stream);
    auto t_all = std::chrono::steady_clock::now();
    nsg_index *ix = new (std::nothrow) nsg_index;
    if (!ix) return NSG_ENOMEM;
    ix->n = n;
    ix->d = d;
    ix->dp = round_up4(d);
    ix->R = R;
    DevBuf<float> base;
    DevBuf<int> adj, deg, knn;
    DevBuf<double> cen, part;
    nsg_status s = padded_copy(base_dev, n, d, ix->dp, base, st);
    cudaError_t e = cudaSuccess;
    if (!s && (e = adj.alloc((size_t)n * R)) != cudaSuccess) s = cuda_fail(e, "alloc adj");
    if (!s && (e = deg.alloc((size_t)n)) != cudaSuccess) s = cuda_fail(e, "alloc deg");
    if (!s && (e = knn.alloc((size_t)n * K)) != cudaSuccess) s = cuda_fail(e, "alloc knn");
    // A1: kNN graph, exact or by nn-descent
    auto t0 = std::chrono::steady_clock::now();
    if (!s && !nnd) s = knn_run(base.p, n, ix->dp, base.p, n, 0, K, 1, knn.p, nullptr, st);
    if (!s && nnd) s = nndescent_run(base.p, n, ix->dp, d, K, *nnd, knn.p, nullptr, &ix->knn_iters, nullptr, st);
    if (!s && (e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(e, "knn");
    ix->ms[0] = (float)since_ms(t0);
    // A2 + A3: centroid and navigating node
    t0 = std::chrono::steady_clock::now();
    int nb = nsg::sm_count() * 4;
    if (!s && (e = part.alloc((size_t)nb * ix->dp)) != cudaSuccess) s = cuda_fail(e, "alloc part");
    if (!s && (e = cen.alloc((size_t)ix->dp)) != cudaSuccess) s = cuda_fail(e, "alloc centroid");
    if (!s && (e = nsg::launch_centroid(base.p, n, ix->dp, part.p, nb, cen.p, st)) != cudaSuccess)
        s = cuda_fail(e, "centroid");
    const int start = (int)(splitmix64(seed) % (uint64_t)n);
    if (!s) s = navigate_run(base.p, n, ix->dp, knn.p, K, cen.p, start, L, &ix->nav, st);
    ix->ms[1] = (float)since_ms(t0);
    // A5 + A6: search-collect-select per node
    if (!s)
        s = collect_prune_all(base.p, n, ix->dp, knn.p, K, ix->nav, L, R, C, adj.p, deg.p, &ix->ms[2],
                              &ix->ms[3], &ix->prune_examined, st);
    knn.alloc(0);  // release the kNN graph before the connectivity pass
    // A7: connectivity
    t0 = std::chrono::steady_clock::now();
    int added = 0, research = 0;
    if (!s) s = connect_run(base.p, n, ix->dp, adj.p, deg.p, R, ix->nav, L, &added, st, &research);
    ix->ms[4] = (float)since_ms(t0);
    ix->n_fixup = added;
    ix->n_fixup_searches = research;
    if (s) {
        destroy(ix);
        return s;
    }
    ix->base = base.release();
    ix->adj = adj.release();
    ix->deg = deg.release();
    s = finish_index(ix, st);
    ix->ms[5] = (float)since_ms(t_all);
    if (s) {
        destroy(ix);
        return s;
    }
    *out = ix;
    return NSG_OK;
}

nsg_status nsg_build(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                     int32_t C, uint64_t seed, void *stream, nsg_index **out) {
    return build_index(base_dev, n, d, K, L, R, C, seed, nullptr, stream, out);
}

nsg_status nsg_build_ex(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                        int32_t C, uint64_t seed, const nsg_nndescent_params *knn_params, void *stream,
                        nsg_index **out) {
    if (knn_params && (!nndescent_params_ok(*knn_params) || knn_params->reverse > K)) {
        if (out) *out = nullptr;
        return NSG_EINVAL;
    }
    return build_index(base_dev, n, d, K, L, R, C, seed, knn_params, stream, out);
}

nsg_status nsg_knn_nndescent(const float *base_dev, int64_t n, int32_t d, int32_t K,
                             const nsg_nndescent_params *params, int32_t *knn_ids_dev, float *knn_d2_dev,
                             int32_t *iters_run, int64_t *last_updates, void *stream) {
    return host_guard([&]() -> nsg_status {
        if (!base_dev || !knn_ids_dev || !params || n < 2 || n >= INT32_MAX || d < 1 ||
            d > 4 * nsg::MAX_DP4_HOST || K < 1 || K >= n || K > 256 || !nndescent_params_ok(*params) ||
            params->reverse > K)
            return NSG_EINVAL;
        cudaStream_t st = S(stream);
        DevBuf<float> tmp;
        const float *view = nullptr;
        nsg_status s = padded_view(base_dev, n, d, tmp, &view, st);
        if (s) return s;
        int it = 0;
        int64_t upd = 0;
        s = nndescent_run(view, n, round_up4(d), d, K, *params, knn_ids_dev, knn_d2_dev, &it, &upd, st);
        if (s) return s;
        if (iters_run) *iters_run = it;
        if (last_updates) *last_updates = upd;
        return NSG_OK;
    });
}

nsg_status nsg_index_from_graph(const float *base_dev, int64_t n, int32_t d, const int32_t *adj_dev,
                                const int32_t *deg_dev, int32_t R, int32_t nav, void *stream,
                                nsg_index **out) {
    return host_guard([&]() -> nsg_status {
        if (!out) return NSG_EINVAL;
        *out = nullptr;
        if (!base_dev || !adj_dev || n < 1 || n >= INT32_MAX || d < 1 || d > 4 * nsg::MAX_DP4_HOST ||
            R < 1 || R > 1024 || nav < 0 || nav >= n)
            return NSG_EINVAL;
        cudaStream_t st = S(stream);
        nsg_status s = check_ids(adj_dev, n * R, n, st);
        if (s) return s;
        nsg_index *ix = new (std::nothrow) nsg_index;
        if (!ix) return NSG_ENOMEM;
        ix->n = n;
        ix->d = d;
        ix->dp = round_up4(d);
        ix->R = R;
        ix->nav = nav;
        DevBuf<float> base;
        DevBuf<int> adj, deg;
        s = padded_copy(base_dev, n, d, ix->dp, base, st);
        cudaError_t e = cudaSuccess;
        if (!s && (e = adj.alloc((size_t)n * R)) != cudaSuccess) s = cuda_fail(e, "alloc adj");
        if (!s && (e = deg.alloc((size_t)n)) != cudaSuccess) s = cuda_fail(e, "alloc deg");
        if (!s && (e = cudaMemcpyAsync(adj.p, adj_dev, sizeof(int) * n * R, cudaMemcpyDeviceToDevice, st)) !=
                      cudaSuccess)
            s = cuda_fail(e, "copy adj");
        if (!s) {
            if (deg_dev) {
                e = cudaMemcpyAsync(deg.p, deg_dev, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) s = cuda_fail(e, "copy deg");
            } else {
                std::vector<int> h((size_t)n * R), dg((size_t)n);
                e = cudaMemcpyAsync(h.data(), adj_dev, sizeof(int) * n * R, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e == cudaSuccess) {
                    for (int64_t v = 0; v < n; ++v) {
                        int c = 0;
                        while (c < R && h[v * R + c] >= 0) ++c;
                        dg[v] = c;
                    }
                    e = cudaMemcpyAsync(deg.p, dg.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                }
                if (e != cudaSuccess) s = cuda_fail(e, "degrees");
            }
        }
        if (s) {
            destroy(ix);
            return s;
        }
        ix->base = base.release();
        ix->adj = adj.release();
        ix->deg = deg.release();
        s = finish_index(ix, st);
        if (s) {
            destroy(ix);
            return s;
        }
        *out = ix;
        return NSG_OK;
    });
}

nsg_status nsg_build_partitioned(const float *base_dev, int64_t n, int32_t d, const int32_t *part_host,
                                 int32_t P, int32_t K, int32_t L, int32_t R, int32_t C, uint64_t seed,
                                 void *stream, nsg_index **out) {
    return host_guard([&]() -> nsg_status {
        if (!out) return NSG_EINVAL;
        *out = nullptr;
        if (!base_dev || !part_host || n < 2 || n >= INT32_MAX || d < 1 || d > 4 * nsg::MAX_DP4_HOST || P < 1 ||
            P > 4096 || K < 1 || L < 1 || L > 1024 || R < 1 || R > 1024 || C < R || C > 4096)
            return NSG_EINVAL;
        // subsets in ascending id, rows of a subset in ascending row order
        std::vector<int64_t> off((size_t)P + 1, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int p = part_host[i];
            if (p < 0 || p >= P) return NSG_EINVAL;
            ++off[(size_t)p + 1];
        }
        for (int p = 0; p < P; ++p) {
            if (off[(size_t)p + 1] < 2) return NSG_EINVAL;  // every subset needs 2 rows
            off[(size_t)p + 1] += off[(size_t)p];
        }
        std::vector<int> perm((size_t)n);
        {
            std::vector<int64_t> fill(off.begin(), off.end() - 1);
            for (int64_t i = 0; i < n; ++i) perm[(size_t)fill[(size_t)part_host[i]]++] = (int)i;
        }
        cudaStream_t st = S(stream);
        auto t_all = std::chrono::steady_clock::now();
        DevBuf<int> perm_d, adj, deg, starts_d;
        DevBuf<float> rows;  // the base in subset order, [n][d]
        NSG_CK(perm_d.alloc((size_t)n));
        NSG_CK(adj.alloc((size_t)n * R));
        NSG_CK(deg.alloc((size_t)n));
        NSG_CK(starts_d.alloc((size_t)P));
        NSG_CK(rows.alloc((size_t)n * d));
        NSG_CK(cudaMemcpyAsync(perm_d.p, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        NSG_CK(nsg::launch_gather_rows(base_dev, n, d, perm_d.p, rows.p, st));
        std::vector<int> starts((size_t)P);
        float ms[5] = {0, 0, 0, 0, 0};
        int64_t fixups = 0, researched = 0, examined = 0;
        for (int p = 0; p < P; ++p) {
            const int64_t o = off[(size_t)p], np = off[(size_t)p + 1] - o;
            const int Kp = (int)std::min<int64_t>(K, np - 1);
            nsg_index *sub = nullptr;
            nsg_status s = nsg_build(rows.p + o * d, np, d, Kp, L, R, C, seed, stream, &sub);
            if (s) return s;
            std::unique_ptr<nsg_index, void (*)(nsg_index *)> hold(sub, destroy);
            NSG_CK(nsg::launch_offset_adj(sub->adj, np, R, (int)o, adj.p + o * R, st));
            NSG_CK(cudaMemcpyAsync(deg.p + o, sub->deg, sizeof(int) * np, cudaMemcpyDeviceToDevice, st));
            NSG_CK(cudaStreamSynchronize(st));
            starts[(size_t)p] = (int)o + sub->nav;
            for (int t = 0; t < 5; ++t) ms[t] += sub->ms[t];
            fixups += sub->n_fixup;
            researched += sub->n_fixup_searches;
            examined += sub->prune_examined;
        }
        NSG_CK(cudaMemcpyAsync(starts_d.p, starts.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
        nsg_index *ix = new (std::nothrow) nsg_index;
        if (!ix) return NSG_ENOMEM;
        std::unique_ptr<nsg_index, void (*)(nsg_index *)> hold(ix, destroy);
        ix->n = n;
        ix->d = d;
        ix->dp = round_up4(d);
        ix->R = R;
        ix->nav = starts[0];
        DevBuf<float> base;
        nsg_status s = padded_copy(rows.p, n, d, ix->dp, base, st);
        if (s) return s;
        NSG_CK(cudaStreamSynchronize(st));
        ix->base = base.release();
        ix->adj = adj.release();
        ix->deg = deg.release();
        ix->parts = P;
        ix->starts = starts_d.release();
        ix->perm = perm_d.release();
        ix->part_off = off;
        for (int t = 0; t < 5; ++t) ix->ms[t] = ms[t];
        ix->n_fixup = fixups;
        ix->n_fixup_searches = researched;
        ix->prune_examined = examined;
        s = finish_index(ix, st);
        if (s) return s;
        ix->ms[5] = (float)since_ms(t_all);
        *out = hold.release();
        return NSG_OK;
    });
}

namespace {

// Validated launch description for nsg_search_ex / nsg_search_trace.
nsg_status make_search(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k, int32_t L,
                       const nsg_search_params *params, int32_t *ids_dev, float *d2_dev, int32_t *n_expand_dev,
                       int32_t *n_dist_dev, int32_t *status_dev, nsg::SearchLaunch &l) {
    if (!idx || k < 1 || L < k || L > NSG_MAX_L || nq < 0 || nq >= INT32_MAX) return NSG_EINVAL;
    if (nq > 0 && (!queries_dev || !ids_dev)) return NSG_EINVAL;
    nsg_search_params p = {0, 0, NSG_PREC_F32, 0, -1, nullptr, 0.5f, 0, 0, 0, 0, 0, 0, 0};
    if (params) p = *params;
    if (p.pool < 0 || p.pool > 2 || (p.pool == 1 && L > 1024)) return NSG_EINVAL;
    l.pool_global = p.pool == 2 || (p.pool == 0 && L > 1024);
    if (p.stage_rows > NSG_STAGE_MAX || (p.stage_rows > 0 && (idx->dp <= 512 || p.stop_model))) return NSG_EINVAL;
    l.stage = p.stage_rows == 0 ? -1 : (p.stage_rows < 0 ? 0 : p.stage_rows);
    if (p.precision < NSG_PREC_F32 || p.precision > NSG_PREC_U8) return NSG_EINVAL;
    if (p.init_random < 0 || p.init_random > L) return NSG_EINVAL;
    if (p.warps_per_query != 0 && p.warps_per_query != 1 && p.warps_per_query != 2 && p.warps_per_query != 4)
        return NSG_EINVAL;
    if (p.precision != NSG_PREC_F32 && !idx->lowp[p.precision]) return NSG_EINVAL;  // nsg_index_prepare first
    if (p.hash_slots > 0 && (p.hash_slots < 64 || (p.hash_slots & (p.hash_slots - 1)) || p.hash_slots > 65536))
        return NSG_EINVAL;
    if (p.stop_model && !(p.stop_threshold > 0.0f && p.stop_threshold < 1.0f)) return NSG_EINVAL;
    if (p.stop_model) {
        l.stop_model = p.stop_model;
        l.stop_logit = std::log(p.stop_threshold / (1.0f - p.stop_threshold));
    }
    l.stop_k = p.stop_k > 0 ? (p.stop_k < L ? p.stop_k : L) : (k < 10 ? k : 10);
    l.stop_min_steps = p.stop_min_steps > 0 ? p.stop_min_steps : 0;
    l.base = idx->base;
    l.n = idx->n;
    l.dp = idx->dp;
    l.adj = idx->adj;
    l.width = idx->R;
    l.start = idx->nav;
    l.queries = queries_dev;
    l.d = idx->d;
    l.nq = nq;
    l.k = k;
    l.L = L;
    l.hash_slots = 0;  // below, once the warps per query are known
    l.max_steps = p.max_steps > 0 ? p.max_steps : nsg::default_steps(L);
    l.warps_per_cta = p.warps_per_cta;
    l.ids = ids_dev;
    l.d2 = d2_dev;
    l.n_expand = n_expand_dev;
    l.n_dist = n_dist_dev;
    l.status = status_dev;
    l.any_capped = nullptr;
    l.init_count = p.init_random;
    l.init_seed = p.init_seed;
    l.warps_per_query = p.warps_per_query > 0 ? p.warps_per_query : nsg::search_auto_wpq(nq, idx->dp, p.precision, L);
    const bool staged = idx->dp > 512 && (p.stage_rows > 0 || (p.stage_rows == 0 && p.precision == NSG_PREC_F32));
    l.hash_slots = p.hash_slots > 0 ? p.hash_slots
                                    : default_search_hash(L, idx->R, nq, l.warps_per_query, staged || p.stop_model);
    if (p.precision != NSG_PREC_F32) {
        l.precision = p.precision;
        l.lowp = idx->lowp[p.precision];
        l.lowp_map = idx->lowp_map[p.precision];
        l.lowp_chunks = idx->lowp_dpl[p.precision] * (p.precision == NSG_PREC_BF16 ? 2 : 1) / 16;
        l.lowp_scale = idx->lowp_scale[p.precision];
        l.lowp_lo = idx->lowp_lo[p.precision];
        // auto: re-rank unless the copy holds every value exactly (then its keys
        // are the FP32 keys); an exact U8 copy still re-ranks a query whose
        // values the 8-bit map rounds
        const int exact = idx->lowp_exact[p.precision];
        l.rerank = p.rerank < 0 ? (!exact ? 1 : (p.precision == NSG_PREC_U8 ? 2 : 0)) : (p.rerank != 0);
    }
    return NSG_OK;
}

// Search launch whose warps draw queries from a device counter: a warp that
// finishes early takes the next query, instead of a fixed share of
// ceil(nq / warps) queries leaving a tail of warps on their last one.  The
// counter is one of the index's kWorkSlots, taken round-robin and zeroed on
// the launch's stream, so calls on one stream are ordered and up to
// kWorkSlots calls may run concurrently on different streams.
// Global-memory pools for a launch that asks for them: the index's slots,
// grown (after the stream has drained) when this L needs more bytes.
nsg_status ensure_gpool_body(const nsg_index *idx, nsg::SearchLaunch &l, cudaStream_t st) {
    if (!l.pool_global) return NSG_OK;
    const int64_t slots = nsg::search_pool_slots();
    const size_t need = (size_t)slots * (size_t)l.L * sizeof(uint64_t);
    std::lock_guard<std::mutex> lock(idx->gpool_mu);
    if (need > idx->gpool_bytes) {
        NSG_CK(cudaStreamSynchronize(st));
        if (idx->gpool) cudaFree(idx->gpool);
        idx->gpool = nullptr;
        idx->gpool_bytes = 0;
        NSG_CK(cudaMalloc(reinterpret_cast<void **>(&idx->gpool), need));
        idx->gpool_bytes = need;
    }
    l.gpool = idx->gpool;
    l.gpool_slots = slots;
    return NSG_OK;
}

nsg_status ensure_gpool(const nsg_index *idx, nsg::SearchLaunch &l, cudaStream_t st) {
    return host_guard([&] { return ensure_gpool_body(idx, l, st); });
}

// The library's own stream-ordered pool for per-call scratch on this device:
// it keeps what it has mapped (release threshold: never), where the default
// pool gives it back at every synchronisation and the next call maps it
// again.  Created once per device, kept until the process exits.
cudaMemPool_t scratch_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

nsg_status launch_dynamic(const nsg_index *idx, nsg::SearchLaunch l, cudaStream_t st) {
    if (nsg_status s = ensure_gpool(idx, l, st)) return s;
    int *ctr = idx->work + (idx->work_next.fetch_add(1, std::memory_order_relaxed) % kWorkSlots);
    NSG_CK(cudaMemsetAsync(ctr, 0, sizeof(int), st));
    l.work = ctr;
    // queries farthest from the navigating node drawn first (the launch's tail
    // is then made of short searches) when the batch has more warps' worth of
    // queries than the GPU holds at once (otherwise every query starts at
    // once); the order's scratch is stream-ordered, so calls on other streams
    // never share it.  Without it the batch runs in its own order.
    void *scratch = nullptr;
    const int64_t resident = (int64_t)nsg::sm_count() * 32;
    const int wpq = l.warps_per_query > 1 ? l.warps_per_query : 1;
    const bool ordered = l.parts <= 1 && l.order == nullptr && l.init_count == 0 && l.nq * wpq > resident;
    cudaMemPool_t pool = ordered ? scratch_pool() : nullptr;
    if (pool && cudaMallocFromPoolAsync(&scratch, nsg::nav_order_scratch_bytes(l.nq), pool, st) == cudaSuccess) {
        int *ord = nullptr;
        if (nsg::launch_nav_order(l.queries, l.nq, l.d, l.base + (int64_t)l.start * l.dp, scratch, &ord, st) ==
            cudaSuccess)
            l.order = ord;
    } else {
        cudaGetLastError();  // an allocation refused is not an error of this call
    }
    const cudaError_t e = nsg::launch_search(l, st);
    if (scratch) cudaFreeAsync(scratch, st);
    NSG_CK(e);
    return NSG_OK;
}

}  // namespace

nsg_status nsg_search_ex(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k,
                         int32_t L, const nsg_search_params *params, int32_t *ids_dev, float *d2_dev,
                         int32_t *n_expand_dev, int32_t *n_dist_dev, int32_t *status_dev, void *stream) {
    nsg::SearchLaunch l;
    nsg_status s = make_search(idx, queries_dev, nq, k, L, params, ids_dev, d2_dev, n_expand_dev, n_dist_dev,
                               status_dev, l);
    if (s || nq == 0) return s;
    return launch_dynamic(idx, l, S(stream));
}

nsg_status nsg_search_partitioned(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k,
                                  int32_t L, const nsg_search_params *params, int32_t *ids_dev, float *d2_dev,
                                  void *stream) {
    return host_guard([&]() -> nsg_status {
        if (!idx || idx->parts < 2 || !idx->starts || !idx->perm || (nq > 0 && !ids_dev)) return NSG_EINVAL;
        if (params && (params->stop_model || params->init_random)) return NSG_EINVAL;
        const int P = idx->parts;
        if (nq < 0 || nq >= INT32_MAX / P) return NSG_EINVAL;
        nsg::SearchLaunch l;
        // units (query, subset); their result rows [nq * P][k] go to scratch
        int32_t *iph = reinterpret_cast<int32_t *>(16);
        nsg_status s = make_search(idx, queries_dev, nq * P, k, L, params, iph, nullptr, nullptr, nullptr,
                                   nullptr, l);
        if (s || nq == 0) return s;
        cudaStream_t st = S(stream);
        std::lock_guard<std::mutex> lock(idx->part_mu);
        const int64_t need = nq * P * (int64_t)k;
        if (need > idx->part_cap) {
            NSG_CK(cudaStreamSynchronize(st));
            if (idx->part_ids) cudaFree(idx->part_ids);
            if (idx->part_d2) cudaFree(idx->part_d2);
            idx->part_ids = nullptr;
            idx->part_d2 = nullptr;
            idx->part_cap = 0;
            NSG_CK(cudaMalloc(reinterpret_cast<void **>(&idx->part_ids), sizeof(int) * need));
            NSG_CK(cudaMalloc(reinterpret_cast<void **>(&idx->part_d2), sizeof(float) * need));
            idx->part_cap = need;
        }
        l.ids = idx->part_ids;
        l.d2 = idx->part_d2;
        l.parts = P;
        l.starts = idx->starts;
        s = launch_dynamic(idx, l, st);
        if (s) return s;
        NSG_CK(nsg::launch_merge_parts(idx->part_ids, idx->part_d2, nq, P, k, idx->perm, k, ids_dev, d2_dev, st));
        return NSG_OK;
    });
}

nsg_status nsg_search_host(const nsg_index *idx, const float *queries_host, int64_t nq, int32_t k, int32_t L,
                           const nsg_search_params *params, int32_t *ids_host, float *d2_host, void *stream) {
    if (!idx || (nq > 0 && (!queries_host || !ids_host))) return NSG_EINVAL;
    // validate with placeholder device pointers (nothing is launched here)
    nsg::SearchLaunch l;
    const float *qph = reinterpret_cast<const float *>(16);
    int *iph = reinterpret_cast<int *>(16);
    nsg_status s = make_search(idx, qph, nq, k, L, params, iph, nullptr, nullptr, nullptr, nullptr, l);
    if (s || nq == 0) return s;
    std::lock_guard<std::mutex> lock(idx->host_mu);
    const int d = idx->d;
    if (nq > idx->host_cap || k > idx->host_k) {
        const int64_t cap = nq > idx->host_cap ? nq : idx->host_cap;
        const int kc = k > idx->host_k ? k : idx->host_k;
        cudaFree(idx->host_q);
        cudaFree(idx->host_ids);
        cudaFree(idx->host_d2);
        idx->host_q = nullptr;
        idx->host_ids = nullptr;
        idx->host_d2 = nullptr;
        idx->host_cap = 0;
        idx->host_k = 0;
        NSG_CK(cudaMalloc(&idx->host_q, sizeof(float) * cap * d));
        NSG_CK(cudaMalloc(&idx->host_ids, sizeof(int) * cap * kc));
        NSG_CK(cudaMalloc(&idx->host_d2, sizeof(float) * cap * kc));
        idx->host_cap = cap;
        idx->host_k = kc;
    }
    if (!idx->host_flag) NSG_CK(cudaMalloc(&idx->host_flag, sizeof(int)));
    // one copy in, one search over the whole batch, one copy out, on the
    // caller's stream.  Splitting the batch over two streams to overlap the
    // copies was measured slower (each smaller launch ends in its own tail of
    // long queries, while the copies are ~1 % of the step on this host link).
    // On any error the stream is still drained before returning, so no copy
    // touches the caller's host buffers after the call.
    cudaStream_t st = S(stream);
    cudaError_t e = cudaMemsetAsync(idx->host_flag, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(idx->host_q, queries_host, sizeof(float) * nq * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        l.queries = idx->host_q;
        l.ids = idx->host_ids;
        l.d2 = d2_host ? idx->host_d2 : nullptr;
        l.any_capped = idx->host_flag;
        s = launch_dynamic(idx, l, st);
    }
    if (e == cudaSuccess && s == NSG_OK)
        e = cudaMemcpyAsync(ids_host, idx->host_ids, sizeof(int) * nq * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && s == NSG_OK && d2_host)
        e = cudaMemcpyAsync(d2_host, idx->host_d2, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st);
    int capped = 0;
    if (e == cudaSuccess && s == NSG_OK)
        e = cudaMemcpyAsync(&capped, idx->host_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = se;
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "nsg_search_host");
    return (capped & 2) ? NSG_ECUDA : capped ? NSG_ESTEPCAP : NSG_OK;  // bit 1: a staged copy never landed
}

}  // extern "C"

struct nsg_plan {
    nsg::SearchLaunch l;
    int *order = nullptr;  // visiting order (longest pool first)
    int *work = nullptr;   // device work counter
    uint64_t *gpool = nullptr;  // global-memory pool slots (the graph keeps the address)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    nsg_plan_info_t info = {0, 0, 0, 0.0f, 0.0f, 1, 1};
};

namespace {

void plan_destroy(nsg_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->gpool) cudaFree(p->gpool);
    if (p->order) cudaFree(p->order);
    if (p->work) cudaFree(p->work);
    delete p;
}

// Validated batched launch with its visiting order (queries sorted by pool
// size, largest first, so the longest searches start first) and work counter.
nsg_status batched_setup_body(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                         const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                         int32_t *ids_dev, float *d2_dev, int32_t *status_dev, nsg::SearchLaunch &l,
                         DevBuf<int> &order, DevBuf<int> &work, cudaStream_t st) {
    if (!k_dev || !L_dev || kmax < 1 || Lmax < kmax) return NSG_EINVAL;
    nsg_status s = make_search(idx, queries_dev, nq, kmax, Lmax, params, ids_dev, d2_dev, nullptr, nullptr,
                               status_dev, l);
    if (s) return s;
    std::vector<int> hL((size_t)nq), ord((size_t)nq);
    NSG_CK(cudaMemcpyAsync(hL.data(), L_dev, sizeof(int) * nq, cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < nq; ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hL[a] > hL[b]; });
    NSG_CK(order.alloc((size_t)nq));
    NSG_CK(work.alloc(1));
    NSG_CK(cudaMemcpyAsync(order.p, ord.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, st));
    NSG_CK(cudaStreamSynchronize(st));
    l.kv = k_dev;
    l.Lv = L_dev;
    l.order = order.p;
    l.work = work.p;
    return NSG_OK;
}

nsg_status batched_setup(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                         const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                         int32_t *ids_dev, float *d2_dev, int32_t *status_dev, nsg::SearchLaunch &l,
                         DevBuf<int> &order, DevBuf<int> &work, cudaStream_t st) {
    return host_guard([&] {
        return batched_setup_body(idx, queries_dev, nq, k_dev, L_dev, kmax, Lmax, params, ids_dev, d2_dev,
                                  status_dev, l, order, work, st);
    });
}

nsg_status batched_run(const nsg::SearchLaunch &l, cudaStream_t st) {
    NSG_CK(cudaMemsetAsync(l.work, 0, sizeof(int), st));
    NSG_CK(nsg::launch_search(l, st));
    return NSG_OK;
}

}  // namespace

extern "C" {

nsg_status nsg_search_batched(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                              const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                              int32_t *ids_dev, float *d2_dev, int32_t *status_dev, void *stream) {
    if (nq == 0 && idx) return NSG_OK;
    cudaStream_t st = S(stream);
    nsg::SearchLaunch l;
    DevBuf<int> order, work;
    nsg_status s = batched_setup(idx, queries_dev, nq, k_dev, L_dev, kmax, Lmax, params, ids_dev, d2_dev,
                                 status_dev, l, order, work, st);
    if (s) return s;
    if ((s = ensure_gpool(idx, l, st))) return s;
    s = batched_run(l, st);
    if (s) return s;
    NSG_CK(cudaStreamSynchronize(st));  // the order / counter scratch is freed on return
    return NSG_OK;
}

nsg_status nsg_plan_create(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                           const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                           int32_t *ids_dev, float *d2_dev, int32_t *status_dev, int32_t autotune, void *stream,
                           nsg_plan **out) {
    if (!out) return NSG_EINVAL;
    *out = nullptr;
    if (nq < 1) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg_plan *p = new (std::nothrow) nsg_plan;
    if (!p) return NSG_ENOMEM;
    DevBuf<int> order, work;
    nsg_status s = batched_setup(idx, queries_dev, nq, k_dev, L_dev, kmax, Lmax, params, ids_dev, d2_dev,
                                 status_dev, p->l, order, work, st);
    if (s) {
        plan_destroy(p);
        return s;
    }
    p->order = order.release();
    p->work = work.release();
    // the plan's own global-memory pool slots (its graph keeps their address):
    // needed above L = 1024, and tried by the autotuner below that
    const bool want_gpool = p->l.pool_global || (autotune && (!params || params->pool == 0));
    if (want_gpool) {
        const int64_t slots = nsg::search_pool_slots();
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p->gpool), (size_t)slots * Lmax * sizeof(uint64_t));
        if (e != cudaSuccess) {
            plan_destroy(p);
            return cuda_fail(e, "plan pool");
        }
        p->l.gpool_slots = slots;
        if (p->l.pool_global) p->l.gpool = p->gpool;
    }
    if (autotune) {  // time each launch shape on the bound batch; keep the fastest
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f, worst = 0.0f;
        int bw = 0, bh = 0, bq = 1, tried = 0, bs = p->l.stage;
        uint64_t *bp = p->l.gpool;
        const bool groups_ok = p->l.stop_model == nullptr;  // the stop kernels run one warp per query
        // pool placement: shared memory where L fits (<= 1024) unless the caller
        // fixed it, global memory when the plan holds slots
        std::vector<uint64_t *> pools;
        if (!p->l.pool_global) pools.push_back(nullptr);
        if (p->gpool) pools.push_back(p->gpool);
        // row gathers: registers and (rows of more than 512 values) staged,
        // unless the caller fixed them
        std::vector<int> stages;
        if (params && params->stage_rows != 0) stages.push_back(p->l.stage);
        else {
            stages.push_back(0);
            if (p->l.dp > 512 && groups_ok) stages.push_back(-1);
        }
        for (int sg : stages)
        for (uint64_t *gp : pools)
        for (int q : {1, 2, 4})
            for (int w : {2, 4, 8})
            for (int h : {512, 1024, 2048}) {
                if (w < q || (q > 1 && !groups_ok)) continue;
                nsg::SearchLaunch t = p->l;
                t.warps_per_cta = w;
                t.hash_slots = h;
                t.warps_per_query = q;
                t.gpool = gp;
                t.stage = sg;
                if (sg < 0 && nsg::search_stage_resolve(t) == 0) continue;  // auto resolves to registers
                if (batched_run(t, st) || cudaStreamSynchronize(st) != cudaSuccess) continue;
                cudaEventRecord(e0, st);
                bool ok = true;
                for (int r = 0; r < 3 && ok; ++r) ok = batched_run(t, st) == NSG_OK;
                cudaEventRecord(e1, st);
                if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= 3.0f;
                ++tried;
                worst = ms > worst ? ms : worst;
                if (ms < best) {
                    best = ms;
                    bw = w;
                    bh = h;
                    bq = q;
                    bp = gp;
                    bs = sg;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (tried) {
            p->l.warps_per_cta = bw;
            p->l.hash_slots = bh;
            p->l.warps_per_query = bq;
            p->l.gpool = bp;
            p->l.stage = bs;
            p->info.best_ms = best;
            p->info.worst_ms = worst;
        }
        p->info.n_tried = tried;
    }
    p->info.warps_per_cta = p->l.warps_per_cta > 0 ? p->l.warps_per_cta : 4;
    p->info.hash_slots = p->l.hash_slots;
    p->info.warps_per_query = p->l.warps_per_query;
    p->info.pool = p->l.gpool ? 2 : 1;
    p->info.stage_rows = nsg::search_stage_resolve(p->l);
    // capture "reset counter + search" once; a run replays it
    s = batched_run(p->l, st);  // sets kernel attributes outside the capture
    cudaError_t e = cudaStreamSynchronize(st);
    if (!s && e != cudaSuccess) s = cuda_fail(e, "plan warm-up");
    cudaStream_t cs = nullptr;
    if (!s && (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) s = cuda_fail(e, "stream");
    if (!s && (e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        s = cuda_fail(e, "begin capture");
    if (!s) {
        nsg_status r = batched_run(p->l, cs);
        e = cudaStreamEndCapture(cs, &p->graph);
        if (r) s = r;
        else if (e != cudaSuccess) s = cuda_fail(e, "end capture");
    }
    if (!s && (e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) s = cuda_fail(e, "instantiate");
    if (cs) cudaStreamDestroy(cs);
    if (s) {
        plan_destroy(p);
        return s;
    }
    *out = p;
    return NSG_OK;
}

nsg_status nsg_plan_run(nsg_plan *plan, void *stream) {
    if (!plan || !plan->exec) return NSG_EINVAL;
    NSG_CK(cudaGraphLaunch(plan->exec, S(stream)));
    return NSG_OK;
}

nsg_status nsg_plan_info(const nsg_plan *plan, nsg_plan_info_t *info) {
    if (!plan || !info) return NSG_EINVAL;
    *info = plan->info;
    return NSG_OK;
}

void nsg_plan_free(nsg_plan *plan) { plan_destroy(plan); }

nsg_status nsg_search_trace(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k, int32_t L,
                            const nsg_search_params *params, int32_t *ids_dev, float *feat_dev,
                            uint8_t *flag_dev, int32_t *steps_dev, int32_t cap, void *stream) {
    if (cap < 1 || (nq > 0 && (!feat_dev || !flag_dev || !steps_dev))) return NSG_EINVAL;
    nsg_search_params p = {0, 0, NSG_PREC_F32, 0, -1, nullptr, 0.5f, 0, 0, 0, 0, 1, 0, 0};
    if (params) p = *params;
    p.stop_model = nullptr;  // traces record the fixed-L search
    nsg::SearchLaunch l;
    nsg_status s = make_search(idx, queries_dev, nq, k, L, &p, ids_dev, nullptr, steps_dev, nullptr, nullptr, l);
    if (s || nq == 0) return s;
    // the traced features count the new neighbours of each expansion, which
    // the visited set's size changes: traces keep the size the stop model's
    // searches use (the full-batch rule)
    if (p.hash_slots <= 0) l.hash_slots = default_search_hash(L, idx->R);
    l.trace_feat = feat_dev;
    l.trace_flag = flag_dev;
    l.trace_cap = cap;
    if ((s = ensure_gpool(idx, l, S(stream)))) return s;
    NSG_CK(nsg::launch_search(l, S(stream)));
    return NSG_OK;
}

nsg_status nsg_stop_train(const float *feat_dev, const uint8_t *flag_dev, const int32_t *steps_dev, int64_t nq,
                          int32_t cap, int32_t iters, float lr, uint64_t seed, float *master_dev, void *model_dev,
                          float *loss_dev, void *stream) {
    if (!feat_dev || !flag_dev || !steps_dev || !master_dev || !model_dev || nq < 1 || cap < 1 || iters < 1 ||
        !(lr > 0.0f))
        return NSG_EINVAL;
    NSG_CK(nsg::run_stop_train(feat_dev, flag_dev, steps_dev, nq, cap, iters, lr, seed, master_dev, model_dev,
                               loss_dev, S(stream)));
    return NSG_OK;
}

nsg_status nsg_index_prepare(nsg_index *idx, int32_t precision, void *stream) {
    if (!idx || precision < NSG_PREC_BF16 || precision > NSG_PREC_U8) return NSG_EINVAL;
    if (idx->lowp[precision]) return NSG_OK;
    cudaStream_t st = S(stream);
    const int epc = precision == NSG_PREC_BF16 ? 8 : 16;  // values per 16-byte chunk
    const int dpl = (idx->d + epc - 1) / epc * epc;
    float scale = 1.0f, lo = 0.0f;
    bool exact_map = true;  // U8: the map is x - lo (integer data of span <= 255)
    DevBuf<unsigned> flags;
    NSG_CK(flags.alloc(4));
    NSG_CK(cudaMemsetAsync(flags.p, 0, 4 * sizeof(unsigned), st));
    if (precision == NSG_PREC_FP8) {  // per-tensor scale: the largest |x| maps to 448 (e4m3 max)
        unsigned bits = 0;
        NSG_CK(nsg::launch_absmax(idx->base, idx->n * idx->dp, flags.p, st));
        NSG_CK(cudaMemcpyAsync(&bits, flags.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
        NSG_CK(cudaStreamSynchronize(st));
        float mx;
        std::memcpy(&mx, &bits, sizeof(mx));
        scale = mx > 0.0f ? 448.0f / mx : 1.0f;
        NSG_CK(cudaMemsetAsync(flags.p, 0, 4 * sizeof(unsigned), st));
    } else if (precision == NSG_PREC_U8) {  // affine map of [min, max] onto 0..255
        unsigned mm[3] = {0xffffffffu, 0u, 0u};
        NSG_CK(cudaMemcpyAsync(flags.p, mm, sizeof(mm), cudaMemcpyHostToDevice, st));
        NSG_CK(nsg::launch_minmax(idx->base, idx->n, idx->dp, idx->d, flags.p, st));
        NSG_CK(cudaMemcpyAsync(mm, flags.p, sizeof(mm), cudaMemcpyDeviceToHost, st));
        NSG_CK(cudaStreamSynchronize(st));
        const float mn = nsg::float_from_order_key(mm[0]), mx = nsg::float_from_order_key(mm[1]);
        const double span = (double)mx - (double)mn;
        lo = mn;
        exact_map = mm[2] == 0 && span <= 255.0;
        scale = exact_map || !(span > 0.0) ? 1.0f : (float)(255.0 / span);
        NSG_CK(cudaMemsetAsync(flags.p, 0, 4 * sizeof(unsigned), st));
    }
    DevBuf<unsigned char> buf;
    NSG_CK(buf.alloc((size_t)idx->n * dpl * (precision == NSG_PREC_BF16 ? 2 : 1)));
    NSG_CK(nsg::launch_to_lowp(idx->base, idx->n, idx->dp, idx->d, precision, scale, lo, buf.p, dpl,
                               reinterpret_cast<int *>(flags.p), st));
    int inexact = 0;
    NSG_CK(cudaMemcpyAsync(&inexact, flags.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    idx->lowp[precision] = buf.release();
    idx->lowp_dpl[precision] = dpl;
    idx->lowp_scale[precision] = scale;
    idx->lowp_lo[precision] = lo;
    // U8 keys are exact only when the integer sum fits FP32 exactly: d * 255^2 < 2^24
    idx->lowp_exact[precision] =
        !inexact && (precision != NSG_PREC_U8 || (exact_map && (int64_t)idx->d * 65025 < (1 << 24)));
    // rows of more than 512 values and at most 2 KB: a tensor map for the
    // staged gathers, four rows per copy (none: one bulk copy per row)
    const int row_bytes = dpl * (precision == NSG_PREC_BF16 ? 2 : 1);
    alignas(64) unsigned char map[128];
    if (idx->dp > 512 && nsg::make_gather_map(map, idx->lowp[precision], idx->n, row_bytes)) {
        DevBuf<unsigned char> dmap;
        NSG_CK(dmap.alloc(sizeof(map)));
        NSG_CK(cudaMemcpyAsync(dmap.p, map, sizeof(map), cudaMemcpyHostToDevice, st));
        NSG_CK(cudaStreamSynchronize(st));
        idx->lowp_map[precision] = dmap.release();
    }
    return NSG_OK;
}

nsg_status nsg_search(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k, int32_t L,
                      int32_t *ids_dev, float *d2_dev, void *stream) {
    if (!idx || k < 1 || L < k || L > NSG_MAX_L || nq < 0 || nq >= INT32_MAX) return NSG_EINVAL;
    if (nq == 0) return NSG_OK;
    if (!queries_dev || !ids_dev) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    nsg::SearchLaunch l;
    l.base = idx->base;
    l.n = idx->n;
    l.dp = idx->dp;
    l.adj = idx->adj;
    l.width = idx->R;
    l.start = idx->nav;
    l.queries = queries_dev;
    l.d = idx->d;
    l.nq = nq;
    l.k = k;
    l.L = L;
    l.max_steps = nsg::default_steps(L);
    l.warps_per_cta = 0;
    l.ids = ids_dev;
    l.d2 = d2_dev;
    l.n_expand = nullptr;
    l.n_dist = nullptr;
    l.status = nullptr;
    l.any_capped = idx->flag;
    l.stage = -1;  // staged row gathers where they pay (FP32 rows of more than 2 KB)
    l.warps_per_query = nsg::search_auto_wpq(nq, idx->dp, NSG_PREC_F32, L);
    l.hash_slots = default_search_hash(L, idx->R, nq, l.warps_per_query, idx->dp > 512);
    l.pool_global = L > 1024;
    NSG_CK(cudaMemsetAsync(idx->flag, 0, sizeof(int), st));
    if (nsg_status ls = launch_dynamic(idx, l, st)) return ls;
    int h = 0;
    NSG_CK(cudaMemcpyAsync(&h, idx->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    NSG_CK(cudaStreamSynchronize(st));
    return (h & 2) ? NSG_ECUDA : h ? NSG_ESTEPCAP : NSG_OK;  // bit 1: a staged copy never landed
}

nsg_status nsg_recall(const int32_t *ids_dev, int32_t ld_ids, const int32_t *gt_dev, int32_t ld_gt,
                      int64_t nq, int32_t k, int32_t *hits_dev, void *stream) {
    if (nq < 0 || k < 1 || ld_ids < k || ld_gt < k) return NSG_EINVAL;
    if (nq == 0) return NSG_OK;
    if (!ids_dev || !gt_dev || !hits_dev) return NSG_EINVAL;
    NSG_CK(nsg::launch_recall(ids_dev, ld_ids, gt_dev, ld_gt, nq, k, hits_dev, S(stream)));
    return NSG_OK;
}

nsg_status nsg_index_info(const nsg_index *idx, nsg_index_info_t *info) {
    if (!idx || !info) return NSG_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->n = idx->n;
    info->d = idx->d;
    info->R = idx->R;
    info->nav = idx->nav;
    info->max_degree = idx->max_degree;
    info->avg_degree = idx->avg_degree;
    info->n_fixup_edges = idx->n_fixup;
    info->device_bytes = (int64_t)idx->n * idx->dp * 4 + (int64_t)idx->n * idx->R * 4 + idx->n * 4 + 16;
    info->has_bf16 = idx->lowp[NSG_PREC_BF16] ? (idx->lowp_exact[NSG_PREC_BF16] ? 2 : 1) : 0;
    info->has_fp8 = idx->lowp[NSG_PREC_FP8] ? (idx->lowp_exact[NSG_PREC_FP8] ? 2 : 1) : 0;
    info->fp8_scale = idx->lowp[NSG_PREC_FP8] ? idx->lowp_scale[NSG_PREC_FP8] : 0.0f;
    info->n_fixup_searches = idx->n_fixup_searches;
    info->has_u8 = idx->lowp[NSG_PREC_U8] ? (idx->lowp_exact[NSG_PREC_U8] ? 2 : 1) : 0;
    info->u8_lo = idx->lowp[NSG_PREC_U8] ? idx->lowp_lo[NSG_PREC_U8] : 0.0f;
    info->u8_scale = idx->lowp[NSG_PREC_U8] ? idx->lowp_scale[NSG_PREC_U8] : 0.0f;
    info->prune_examined = idx->prune_examined;
    for (int p = 1; p <= 3; ++p)
        if (idx->lowp[p]) info->device_bytes += (int64_t)idx->n * idx->lowp_dpl[p] * (p == 1 ? 2 : 1);
    info->ms_knn = idx->ms[0];
    info->ms_centroid_nav = idx->ms[1];
    info->ms_collect = idx->ms[2];
    info->ms_prune = idx->ms[3];
    info->ms_connect = idx->ms[4];
    info->ms_total = idx->ms[5];
    info->parts = idx->parts;
    info->knn_iters = idx->knn_iters;
    if (idx->parts > 1) info->device_bytes += (int64_t)idx->n * 4 + idx->parts * 4;
    return NSG_OK;
}

nsg_status nsg_index_graph(const nsg_index *idx, int32_t *adj_dev, int32_t *deg_dev, void *stream) {
    if (!idx) return NSG_EINVAL;
    cudaStream_t st = S(stream);
    if (adj_dev)
        NSG_CK(cudaMemcpyAsync(adj_dev, idx->adj, sizeof(int) * idx->n * idx->R, cudaMemcpyDeviceToDevice, st));
    if (deg_dev) NSG_CK(cudaMemcpyAsync(deg_dev, idx->deg, sizeof(int) * idx->n, cudaMemcpyDeviceToDevice, st));
    return NSG_OK;
}

static const char kMagic[8] = {'N', 'S', 'G', 'G', 'B', '3', '0', '0'};

nsg_status nsg_save(const nsg_index *idx, const char *path) {
    return host_guard([&]() -> nsg_status {
        if (!idx || !path || idx->parts > 1) return NSG_EINVAL;
        const int64_t n = idx->n;
        std::vector<int> deg((size_t)n), adj((size_t)n * idx->R);
        std::vector<float> base((size_t)n * idx->d);
        NSG_CK(cudaMemcpy(deg.data(), idx->deg, sizeof(int) * n, cudaMemcpyDeviceToHost));
        NSG_CK(cudaMemcpy(adj.data(), idx->adj, sizeof(int) * n * idx->R, cudaMemcpyDeviceToHost));
        NSG_CK(cudaMemcpy2D(base.data(), sizeof(float) * idx->d, idx->base, sizeof(float) * idx->dp,
                            sizeof(float) * idx->d, n, cudaMemcpyDeviceToHost));
        FILE *f = std::fopen(path, "wb");
        if (!f) return NSG_EIO;
        int32_t hdr[4] = {1, idx->d, idx->R, idx->nav};
        bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, 4, 1, f) == 1 &&
                  std::fwrite(&n, 8, 1, f) == 1 && std::fwrite(&hdr[1], 4, 3, f) == 3 &&
                  std::fwrite(deg.data(), 4, deg.size(), f) == deg.size() &&
                  std::fwrite(adj.data(), 4, adj.size(), f) == adj.size() &&
                  std::fwrite(base.data(), 4, base.size(), f) == base.size();
        ok = (std::fclose(f) == 0) && ok;
        return ok ? NSG_OK : NSG_EIO;
    });
}

nsg_status nsg_load(const char *path, void *stream, nsg_index **out) {
    return host_guard([&]() -> nsg_status {
        if (!path || !out) return NSG_EINVAL;
        *out = nullptr;
        std::unique_ptr<FILE, int (*)(FILE *)> f(std::fopen(path, "rb"), &std::fclose);
        if (!f) return NSG_EIO;
        char magic[8];
        int32_t ver = 0, hdr[3] = {0, 0, 0};
        int64_t n = 0;
        const bool ok = std::fread(magic, 1, 8, f.get()) == 8 && std::fread(&ver, 4, 1, f.get()) == 1 &&
                        std::fread(&n, 8, 1, f.get()) == 1 && std::fread(hdr, 4, 3, f.get()) == 3;
        if (!ok) return NSG_EIO;
        if (std::memcmp(magic, kMagic, 8) != 0 || ver != 1 || n < 1 || n >= INT32_MAX || hdr[0] < 1 ||
            hdr[0] > 4 * nsg::MAX_DP4_HOST || hdr[1] < 1 || hdr[1] > 1024 || hdr[2] < 0 || hdr[2] >= n)
            return NSG_EFORMAT;
        const int d = hdr[0], R = hdr[1], nav = hdr[2];
        // the header must describe exactly the bytes that follow it (checked
        // before anything of that size is allocated)
        const long at = std::ftell(f.get());
        const int64_t want = (int64_t)at + 4 * (n + n * (int64_t)R + n * (int64_t)d);
        if (at < 0 || std::fseek(f.get(), 0, SEEK_END) != 0 || (int64_t)std::ftell(f.get()) != want ||
            std::fseek(f.get(), at, SEEK_SET) != 0)
            return NSG_EFORMAT;
        std::vector<int> deg((size_t)n), adj((size_t)n * R);
        std::vector<float> base((size_t)n * d);
        if (std::fread(deg.data(), 4, deg.size(), f.get()) != deg.size() ||
            std::fread(adj.data(), 4, adj.size(), f.get()) != adj.size() ||
            std::fread(base.data(), 4, base.size(), f.get()) != base.size())
            return NSG_EFORMAT;
        f.reset();
        for (int64_t v = 0; v < n; ++v) {
            if (deg[v] < 0 || deg[v] > R) return NSG_EFORMAT;
            for (int t = 0; t < R; ++t) {
                const int x = adj[v * R + t];
                if (x < -1 || x >= n) return NSG_EFORMAT;
            }
        }
        cudaStream_t st = S(stream);
        DevBuf<float> db;
        DevBuf<int> da, dd;
        NSG_CK(db.alloc(base.size()));
        NSG_CK(da.alloc(adj.size()));
        NSG_CK(dd.alloc(deg.size()));
        NSG_CK(cudaMemcpyAsync(db.p, base.data(), 4 * base.size(), cudaMemcpyHostToDevice, st));
        NSG_CK(cudaMemcpyAsync(da.p, adj.data(), 4 * adj.size(), cudaMemcpyHostToDevice, st));
        NSG_CK(cudaMemcpyAsync(dd.p, deg.data(), 4 * deg.size(), cudaMemcpyHostToDevice, st));
        NSG_CK(cudaStreamSynchronize(st));
        return nsg_index_from_graph(db.p, n, d, da.p, dd.p, R, nav, stream, out);
    });
}

void nsg_free(nsg_index *idx) { destroy(idx); }

}  // extern "C"
