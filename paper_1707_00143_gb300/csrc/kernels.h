// kernels.h -- host-side launchers of the NSG kernels (internal to libnsg).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace nsg {

constexpr int MAX_DP4_HOST = 512;  // largest supported row: 2048 floats

// Step cap of a search with pool size L when the caller sets none: far above
// any expansion count Alg. 1 reaches on a graph (each step checks one of at
// most L pool entries, and an entry is only replaced by a closer one), so it
// only ends a search on a corrupt graph.
inline int default_steps(int L) { return 16 * L + 4096; }

// Search on a fixed-width graph (Alg. 1 from `start`), one warp per query.
struct SearchLaunch {
    const float *base;  // [n][dp] padded, 16-byte aligned
    int64_t n;
    int dp;
    const int *adj;  // [n][width]
    int width;
    int start;
    const float *queries;  // [nq][d]
    int d;
    int64_t nq;
    int k, L;
    int hash_slots, max_steps, warps_per_cta;
    int warps_per_query = 1;  // 1, 2 or 4 warps share a query (search_group_kernel)
    int *ids;
    float *d2;
    int *n_expand, *n_dist, *status;
    int *any_capped;  // device flag, nullable
    // precision forms: traversal on a BF16 / FP8 copy, FP32 re-rank of the pool
    int precision = 0;  // 0 FP32, 1 BF16, 2 FP8-e4m3, 3 U8
    const void *lowp = nullptr;
    int lowp_chunks = 0;  // 16-byte chunks per low-precision row
    float lowp_scale = 1.0f;
    float lowp_lo = 0.0f;  // U8: offset of the 8-bit map
    int rerank = 0;        // 1: always; U8 with 2: only queries the 8-bit map rounds
    // learned early termination (FP16 MLP parameters, nullptr = none) and traces
    const void *stop_model = nullptr;
    float stop_logit = 0.0f;
    int stop_k = 10, stop_min_steps = 0;
    float *trace_feat = nullptr;           // [nq][trace_cap][8]
    unsigned char *trace_flag = nullptr;   // [nq][trace_cap]
    int trace_cap = 0;
    // batched uneven queries: per-query k / L (k, L are then the maxima),
    // visiting order, device work counter (reset before each launch)
    const int *kv = nullptr, *Lv = nullptr, *order = nullptr;
    int *work = nullptr;
    // random initial pool of init_count seeded draws (0: start at `start`)
    int init_count = 0;
    uint64_t init_seed = 0;
    // partitioned search: nq counts (query, subset) units, unit t searches
    // query t / parts from starts[t % parts] and writes output row t
    int parts = 1;
    const int *starts = nullptr;
    // pool placement: shared memory (gpool == nullptr, L <= 1024) or one slot
    // of L keys per resident warp (group) in global memory, gpool_slots slots
    int pool_global = 0;
    uint64_t *gpool = nullptr;
    int64_t gpool_slots = 0;
    // staged row gathers for rows of more than 512 values (stage.cuh): 0 off,
    // > 0 that many rows in flight per warp (at most 32), < 0 chosen by the
    // launch (search_stage_slots); lowp_map: a device tensor map over the
    // low-precision rows (make_gather_map) -- they are then gathered four
    // per copy -- or nullptr
    int stage = 0;
    const void *lowp_map = nullptr;
};
// Approximate kNN graph by nn-descent (nndescent.cu).  base [n][dp] padded
// rows; ids [n][K] out, d2 [n][K] out (nullable); scratch: at least
// nndescent_scratch_bytes(n, K, S, Sr) bytes, 16-byte aligned.  Synchronises
// the stream once per iteration (the stopping rule reads the update count).
struct NnDescentLaunch {
    const float *base;
    int64_t n;
    int dp;
    int K, S, Sr, iters;
    float delta;
    uint64_t seed;
    int *ids;
    float *d2;
    void *scratch;
    int *iters_run;         // host, nullable
    int64_t *last_updates;  // host, nullable
    // an 8-bit copy of the rows (x - u8_lo, u8_chunks 16-byte chunks per row)
    // that holds every distance exactly, or nullptr; d = the row's values
    const void *u8 = nullptr;
    int u8_chunks = 0, d = 0;
    float u8_lo = 0.0f;
};
size_t nndescent_scratch_bytes(int64_t n, int K, int S, int Sr);
cudaError_t launch_nndescent(const NnDescentLaunch &l, cudaStream_t st);

// Resident warps (groups) of any search launch on this device: an upper bound
// on the global-memory pool slots a launch uses (the search kernels hold at
// most 32 warps per SM).
int64_t search_pool_slots();
// Shared memory per warp of the fixed-L search kernels (pool of L keys in
// shared memory, adjacency width rounded to W, H visited slots, no re-rank list).
// Slots per warp the launch gives the staged gathers of rows of `row_bytes`
// when `stage` < 0 (0: the register gather).
int search_stage_slots(int row_bytes);
// Warps per query when the caller leaves them to the library: `units` search
// units (queries, or query-subset pairs) with pools of L keys on rows of `dp`
// padded values in traversal precision `precision`.
int search_auto_wpq(int64_t units, int dp, int precision, int L);
// Rows per warp launch_search gives the staged gathers of `l` (0: none), and
// the ring they take: slots and bytes per slot.
int search_stage_resolve(const SearchLaunch &l);
void stage_layout(const SearchLaunch &l, int nb, int *slots, int *slot_bytes);
// Encode (host) a 2-D tensor map over `n` rows of `row_bytes` (a multiple of
// 16, at most 2048) at `rows` for the staged four-row gathers: 8-byte
// elements, one box = one whole row.  `map` holds 128 bytes.  false: the
// driver's encoder is unavailable or the rows do not qualify.
bool make_gather_map(void *map, const void *rows, int64_t n, int row_bytes);
size_t search_warp_smem_bytes(int L, int W, int H);
cudaError_t launch_search(const SearchLaunch &a, cudaStream_t st);
// Visiting order of nq queries [nq][d] for a work-queue launch: farthest from
// the navigating node's row first (bucketed; the results do not depend on
// it).  scratch: nav_order_scratch_bytes(nq) bytes, 4-byte aligned; *order
// points into it.
size_t nav_order_scratch_bytes(int64_t nq);
cudaError_t launch_nav_order(const float *queries, int64_t nq, int d, const float *nav_row, void *scratch,
                             int **order, cudaStream_t st);

// Partition-and-merge: per query, the union of `parts` sorted result lists
// (ids_in [nq][parts][k_in], positions in the partitioned index, -1 padded;
// d2_in likewise) mapped to row ids through perm and cut to the k smallest
// (distance, row id) keys: ids_out [nq][k], d2_out [nq][k], -1 / +inf padded.
cudaError_t launch_merge_parts(const int *ids_in, const float *d2_in, int64_t nq, int parts, int k_in,
                               const int *perm, int k, int *ids_out, float *d2_out, cudaStream_t st);
// rows of base [n][d] in the order of perm: out[i] = base[perm[i]]
cudaError_t launch_gather_rows(const float *base, int64_t n, int d, const int *perm, float *out, cudaStream_t st);
// adjacency rows of one subset, shifted to its place in the partitioned
// index: out[v][j] = in[v][j] + offset (or -1) for v < nv
cudaError_t launch_offset_adj(const int *in, int64_t nv, int R, int offset, int *out, cudaStream_t st);

// Training of the early-termination MLP on search traces (full-batch Adam).
// feat [nq][cap][8], flag [nq][cap], steps [nq]; label of step t of query q =
// no later step of q changed its first k pool entries.  model_out: FP16
// parameters (w1[64][8], b1[64], w2[64], b2); master: FP32 copy [641] (in/out
// when init == 0).  loss_out (device, nullable): [iters] mean BCE per iteration.
cudaError_t run_stop_train(const float *feat, const unsigned char *flag, const int *steps, int64_t nq, int cap,
                           int iters, float lr, uint64_t seed, float *master, void *model_out, float *loss_out,
                           cudaStream_t st);

// Largest |x| over `count` floats (bits of a non-negative float, atomicMax).
cudaError_t launch_absmax(const float *x, int64_t count, unsigned *out_bits, cudaStream_t st);
// Order-preserving keys of min x and max x (out[0], out[1]; start them at
// 0xffffffff and 0) and out[2] |= 1 when some x is not an integer.
cudaError_t launch_minmax(const float *x, int64_t n, int dp, int d, unsigned *out, cudaStream_t st);
// (key of f: sign bit set -> all bits flipped, else the sign bit set)
inline float float_from_order_key(unsigned k) {
    unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
    memcpy(&f, &b, 4);
    return f;
}
// [n][dp] FP32 -> [n][dpl] BF16 (precision 1), FP8-e4m3 of x*scale (precision 2)
// or U8 of clamp(rint((x - lo) * scale), 0, 255) (precision 3), zero padded;
// *inexact is raised when some value does not survive the round trip.
cudaError_t launch_to_lowp(const float *src, int64_t n, int dp, int d, int precision, float scale, float lo,
                           void *dst, int dpl, int *inexact, cudaStream_t st);

// Search-and-collect on the kNN graph for nodes v0..v0+nv-1.
struct CollectLaunch {
    const float *base;  // [n][dp]
    int64_t n;
    int dp;
    const int *knn;  // [n][K]
    int K, nav, L, C;
    int64_t v0, nv;
    int hash_slots, max_steps;
    int *cand_ids;
    float *cand_d2;
    int *cand_count;
    int *status;
};
cudaError_t launch_collect(const CollectLaunch &a, cudaStream_t st);

// MRNG edge selection for nodes v0..v0+nv-1.
struct PruneLaunch {
    const float *base;  // [n][dp]
    int64_t n;
    int dp;
    const int *cand_ids;
    const float *cand_d2;
    const int *cand_count;  // nullptr: every row holds C candidates
    int C, R;
    int64_t v0, nv;
    int *adj;
    int *deg;
    unsigned long long *examined = nullptr;  // nullable: += candidates examined over all nodes
};
cudaError_t launch_prune(const PruneLaunch &a, cudaStream_t st);

// Centroid in FP64: partial sums per block then an ordered final sum.
cudaError_t launch_centroid(const float *base, int64_t n, int d, double *partial, int nblocks,
                            double *c, cudaStream_t st);

// Navigating node search (single warp, FP64 distances to the centroid).
cudaError_t launch_navigate(const float *base, int64_t n, int d, const int *knn, int K,
                            const double *c, int start, int L, uint32_t *visited_bits,
                            int max_steps, int *nav_out, int *status, cudaStream_t st);

// BFS helpers and the connectivity pass.
cudaError_t launch_bfs_seed(uint32_t *reached, int root, int *frontier, int *count, cudaStream_t st);
cudaError_t launch_bfs_level(const int *adj, int R, const int *frontier, int nf, int *next,
                             int *next_count, uint32_t *reached, cudaStream_t st);
struct ConnectLaunch {
    const float *base;  // [n][dp]
    int64_t n;
    int dp;
    int *adj;  // [n][R], edited in place
    int *deg;
    int R, nav, L;
    int hash_slots, max_steps;
};
// Whole connectivity pass (reach from nav, then speculate/commit fix-up
// batches).  out = {edges added, status, any search capped, re-searches}.
// Allocates its scratch and synchronises the stream.
cudaError_t run_connect(const ConnectLaunch &a, int out[4], cudaStream_t st);

// Precision hits per query (Eq. 1).
cudaError_t launch_recall(const int *ids, int ld_ids, const int *gt, int ld_gt, int64_t nq, int k,
                          int *hits, cudaStream_t st);

// Exact FP32 brute-force k nearest neighbours (serial scan on CUDA cores).
// self_join: queries are the base rows q0.. and each row's own id is skipped.
struct KnnLaunch {
    const float *base;  // [n][dp]
    int64_t n;
    int dp;
    const float *queries;  // [nq][dp]
    int64_t nq;
    int64_t q0;  // id of query 0 when self_join
    int k;
    int self_join;
    int *ids;
    float *d2;
};
cudaError_t launch_knn_direct(const KnnLaunch &a, cudaStream_t st);

// Tensor-core kNN (BF16 GEMM + fused top-k) when the data allows an exact
// answer (integer values 0..255, d <= 128, k <= 256): *used = 1 when it ran,
// 0 when it does not apply (nothing written).  Synchronises the stream.
cudaError_t launch_knn_tc(const KnnLaunch &a, int *used, cudaStream_t st);

// Exact FP32 re-rank: for query i, the k smallest (d2, id) among the KL
// candidate ids cand[i][..] (-1 = none) into a.ids / a.d2.
cudaError_t launch_knn_rerank(const KnnLaunch &a, const int *cand, int KL, cudaStream_t st);

// Padding copy [n][d] -> [n][dp] (zeros in the pad).
cudaError_t launch_pad_rows(const float *src, int64_t n, int d, float *dst, int dp, cudaStream_t st);

// Remember a CUDA error for nsg_last_cuda_error() (calling thread).
void record_cuda_error(cudaError_t e, const char *what);

// Device properties cached per device.
int sm_count();
size_t smem_optin();
size_t smem_per_sm();

}  // namespace nsg
