/*
 * nsg.h -- C ABI of the GB300 (sm_103a) hot path of the Navigating
 * Spreading-out Graph (NSG; Fu, Xiang, Wang, Cai).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Distances are SQUARED l2 (Section 2 defines delta as the l2 distance;
 *    the method only ever compares distances, so squaring changes nothing).
 *  - "Key order" is (squared distance, id) ascending: the distance order
 *    that Alg. 1 keeps its pool in and Alg. 2 sorts candidates by, with the
 *    lower-index tie rule of the MRNG definition (Section 3.3) applied to
 *    every tie.
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *    tensors); *_host are host pointers.  Matrices are dense row-major.
 *    The caller owns every buffer it passes in; an nsg_index owns only what
 *    it allocated itself and frees it in nsg_free().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Unless stated otherwise a call only enqueues work on that
 *    stream and returns; outputs are valid once the stream reaches them.
 *  - Arguments are validated before anything is launched; a violation
 *    returns NSG_EINVAL and touches nothing.  No call throws, aborts or
 *    exits.  Ids are int32 (n < 2^31).  Unused output slots are filled with
 *    id -1 and distance +inf.
 *  - Every device loop has an iteration cap; hitting it never hangs the GPU:
 *    the affected query reports NSG_ESTEPCAP in its status slot and keeps
 *    the partial result.
 */
#ifndef NSG_H
#define NSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NSG_OK = 0,
    NSG_EINVAL = -1,    /* invalid argument; nothing was launched */
    NSG_ENOMEM = -2,    /* device or host allocation failed */
    NSG_ECUDA = -3,     /* a CUDA runtime call failed (see nsg_last_cuda_error) */
    NSG_ESTEPCAP = -4,  /* a search hit its step cap (partial result kept) */
    NSG_EDEGREE = -5,   /* connectivity pass: no reached node has a free slot */
    NSG_EIO = -6,       /* file could not be opened / read / written */
    NSG_EFORMAT = -7    /* file is not an index written by nsg_save */
} nsg_status;

typedef struct nsg_index nsg_index; /* opaque; owns its device memory */

/* Traversal precision of the search.  The final pool is re-ranked on the FP32
 * rows whenever the copy's distances can differ from the FP32 ones (see
 * nsg_search_params.rerank).  NSG_PREC_U8 is an 8-bit affine copy with integer
 * arithmetic (exact on integer data spanning at most 256 values). */
typedef enum { NSG_PREC_F32 = 0, NSG_PREC_BF16 = 1, NSG_PREC_FP8 = 2, NSG_PREC_U8 = 3 } nsg_precision;

typedef struct {
    int32_t max_steps;     /* expansion cap per query; <= 0 -> 16*L + 4096 */
    int32_t hash_slots;    /* visited-hash slots per query (power of 2, 64..65536); <= 0 -> auto:
                              a batch that leaves the SMs short of warps (and stages no rows,
                              has no stop model) takes the largest set up to 4096 (8192 above
                              L = 1024) whose query regions still fit one wave; otherwise 1024
                              when the search still holds 32 warps per SM with it (small
                              pools), else 512; 2048 above L = 1024.  The same results at any
                              size (a forgotten node is measured again) */
    int32_t precision;     /* nsg_precision of the traversal distances */
    int32_t warps_per_cta; /* <= 0 -> auto */
    int32_t rerank;        /* BF16/FP8/U8: re-rank the final pool with FP32 rows (1), not (0),
                              or only when the copy is lossy (-1); U8 with -1 also
                              re-ranks a query whose values the 8-bit map rounds */
    const void *stop_model; /* learned early termination: NSG_STOP_PARAMS FP16 values on the
                               device (see nsg_stop_train), or NULL for the fixed-L search */
    float stop_threshold;  /* stop once the model's probability exceeds this (0..1) */
    int32_t stop_k;        /* result size the stop rule protects (<= 0 -> min(k, 10)) */
    int32_t stop_min_steps; /* never stop before this many expansions; the rule is
                               evaluated at min_steps, min_steps + 4, min_steps + 8, ... */
    int32_t init_random;   /* > 0: the pool starts as the set of this many seeded random
                              nodes (<= L) instead of the navigating node: query q draws
                              splitmix64(init_seed + q * 0x9e3779b97f4a7c15 + j) mod n,
                              j < init_random (NSG-Naive's random initialisation) */
    uint64_t init_seed;
    int32_t warps_per_query; /* 1, 2 or 4 warps share each query: the same steps and
                                results, more rows in flight per expansion (not with a
                                stop model or a trace, which run 1).  0 auto: for FP32
                                rows of more than 2 KB 4 (L <= 1024) or 2; else 1 above
                                L = 1024, and 4, 2 or 1 as the batch leaves each SM fewer
                                than 2, fewer than 8, or more queries */
    int32_t pool;          /* where each query's pool of L keys lives: 0 auto (shared memory
                              up to L = 1024, global memory above), 1 shared memory
                              (L <= 1024), 2 global memory (L <= NSG_MAX_L: one L2-resident
                              slot per resident warp, owned by the index -- or by the plan
                              for nsg_plan_create -- and grown on demand; calls with global
                              pools on one index on different streams at once race on it).
                              The same steps and results either way. */
    int32_t stage_rows;    /* how a warp gathers the base rows it measures, for rows of more
                              than 512 values (d > 512): 0 auto, < 0 through registers (a few
                              rows in flight per warp), 1..NSG_STAGE_MAX staged: each warp
                              copies up to that many rows at once into a ring of shared-memory
                              slots with the bulk-copy (TMA) engine and measures them there
                              (fewer where one query's warps would not fit in a block; the
                              BF16 / FP8 / U8 copies of rows of at most 2 KB four rows per
                              copy, a tile::gather4 through a tensor map that
                              nsg_index_prepare encodes).
                              Auto stages traversal rows of more than 2 KB (FP32 rows of more
                              than 512 values) with 4 slots: bulk copies of rows picked at
                              random complete about one after another, so staging beats the
                              register gather only where that gather holds few rows.  The
                              same steps and results either way.  Staging
                              is refused (NSG_EINVAL) for d <= 512 and with a stop model or a
                              trace.  A staged copy that has not landed after 4 s (a fault,
                              never expected) ends its warp's queries with status NSG_ECUDA. */
} nsg_search_params;

/* Most rows a staged gather holds in flight per warp (nsg_search_params.stage_rows). */
#define NSG_STAGE_MAX 32

/* Largest pool size L of any search (global-memory pools; 1024 in shared memory). */
#define NSG_MAX_L 8192

/* Parameters of the early-termination MLP (8 features -> 64 ReLU -> 1):
 * w1[64][8], b1[64], w2[64], b2 in this order.  The features, formed before
 * each expansion from the pool S (size |S|, k = stop_k, i = position of the
 * entry about to be expanded, t = expansions so far):
 *   0  min(t / L, 4) / 4            4  log2(1 + steps since the first k changed) / 8
 *   1  d(S[0]) / d(S[k-1])          5  i / L
 *   2  min(d(S[k-1]) / d(S[i]), 4)  6  new neighbours at the last expansion / R
 *   3  d(S[k-1]) / d(S[|S|-1])      7  1 if the last expansion changed the first k */
#define NSG_STOP_FEATURES 8
#define NSG_STOP_PARAMS 641

typedef struct {
    int64_t n;             /* base rows */
    int32_t d;             /* dimension */
    int32_t R;             /* adjacency width = max out-degree */
    int32_t nav;           /* navigating node */
    int32_t max_degree;    /* largest out-degree present */
    double avg_degree;     /* mean out-degree (AOD of Table 2) */
    int64_t n_fixup_edges; /* edges added by the connectivity pass */
    int64_t device_bytes;  /* device memory held by the index */
    int32_t has_bf16;      /* BF16 copy: 0 none, 1 lossy, 2 every value exact */
    int32_t has_fp8;       /* FP8-e4m3 copy: 0 none, 1 lossy, 2 every value exact */
    float fp8_scale;       /* x_fp8 = x * fp8_scale (0 when absent) */
    /* build phase wall times in milliseconds (0 when not built here) */
    float ms_knn, ms_centroid_nav, ms_collect, ms_prune, ms_connect, ms_total;
    int64_t n_fixup_searches; /* fix-ups whose speculative search was stale and ran again */
    int32_t has_u8;        /* 8-bit copy: 0 none, 1 lossy, 2 every value and distance exact */
    float u8_lo, u8_scale; /* x_u8 = clamp(rint((x - u8_lo) * u8_scale), 0, 255) */
    int64_t prune_examined; /* candidates the MRNG edge selection examined over all nodes
                               (0 when not built here): per node, every candidate up to the
                               one that filled the row (R kept) or all of them */
    int32_t parts;          /* subsets of a partitioned index (1: a single graph) */
    int32_t knn_iters;      /* nn-descent iterations of the kNN stage (0: exact kNN) */
} nsg_index_info_t;

/* Human-readable name of a status code (static string). */
const char *nsg_status_str(nsg_status s);
/* Text of the last CUDA error seen by this library on the calling thread. */
const char *nsg_last_cuda_error(void);

/* ---------------------------------------------------------------------------
 * A1. Brute-force kNN (serial scan, Section 4.1.2 item 1; Alg. 2 input G).
 *
 * nsg_knn_init: for every base row i, the K nearest OTHER rows in key order
 *   (self excluded by id, so duplicate points stay neighbours).
 *   base_dev [n][d] f32; knn_ids_dev [n][K] i32 out; knn_d2_dev [n][K] f32 out
 *   (nullable).  Requires 1 <= K < n, d >= 1.  Uses tensor cores where the
 *   data allows an exact answer, else an exact FP32 scan.  Allocates scratch.
 *   Environment: NSG_KNN_ENGINE=scan forces the FP32 scan;
 *   NSG_KNN_CHUNK_TILES=t sets the tensor-core form's base chunk (t tiles of
 *   128 rows per launch; default ~48 MB of BF16 rows); the chunk size does
 *   not change results.
 * nsg_knn_query: the k nearest base rows of each query (ground truth):
 *   queries_dev [nq][d]; ids_dev [nq][k]; d2_dev [nq][k] nullable; k <= n.
 * ------------------------------------------------------------------------- */
nsg_status nsg_knn_init(const float *base_dev, int64_t n, int32_t d, int32_t K,
                        int32_t *knn_ids_dev, float *knn_d2_dev, void *stream);
nsg_status nsg_knn_query(const float *base_dev, int64_t n, int32_t d, const float *queries_dev,
                         int64_t nq, int32_t k, int32_t *ids_dev, float *d2_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Approximate kNN graph by nn-descent (Section 3.5 (ii): the build starts
 *   from an approximate kNN graph; Section 3.6's indexing-complexity
 *   paragraph: built with Dong, Charikar and Li's nn-descent for the
 *   million-scale sets).  The published method, deterministic: node v starts
 *   from the first K distinct ids != v among splitmix64(seed + v *
 *   0x9e3779b97f4a7c15 + t) mod n (t = 0, 1, ...), all flagged new; each
 *   iteration samples the first `sample` new and `sample` old entries of
 *   every list (key order; the sampled new ones become old), keeps for every
 *   node the `reverse` nearest of the nodes that sampled it (new and old
 *   separately), joins NEW(v) = new samples u new reverse samples with itself
 *   and with OLD(v) (old samples u old reverse samples, minus NEW(v)), and
 *   cuts every list to the K smallest keys of itself and what it was offered
 *   (entries not in it before are flagged new).  It stops after `iters`
 *   iterations or once an iteration changes at most delta * n * K entries.
 *   The result depends on the inputs alone; on integer data it equals the
 *   CPU oracle's bit for bit (integer data spanning at most 256 values with
 *   d * 255^2 < 2^24 are measured on an 8-bit copy of the rows made for the
 *   call: the same exact distances, a quarter of the bytes).  Recall against
 *   the exact graph is the caller's to measure.
 * nsg_knn_nndescent: knn_ids_dev [n][K] i32 out, knn_d2_dev [n][K] f32 out
 *   (nullable), sorted by key; iters_run / last_updates (host, nullable).
 *   1 <= K < n, K <= 256.  Allocates scratch; synchronises once per
 *   iteration.
 * nsg_build_ex: nsg_build whose kNN stage (A1) is this nn-descent when
 *   knn_params is non-NULL (the exact kNN otherwise).
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t sample;  /* new (and old) entries sampled per list per iteration, 1..256 */
    int32_t reverse; /* reverse samples kept per node (new and old each), 0..K */
    int32_t iters;   /* iteration cap */
    float delta;     /* stop once an iteration changes <= delta * n * K entries */
    uint64_t seed;   /* initial random lists */
} nsg_nndescent_params;

nsg_status nsg_knn_nndescent(const float *base_dev, int64_t n, int32_t d, int32_t K,
                             const nsg_nndescent_params *params, int32_t *knn_ids_dev, float *knn_d2_dev,
                             int32_t *iters_run, int64_t *last_updates, void *stream);
nsg_status nsg_build_ex(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                        int32_t C, uint64_t seed, const nsg_nndescent_params *knn_params, void *stream,
                        nsg_index **out);

/* ---------------------------------------------------------------------------
 * A2. Centroid (Alg. 2, first step): c_j = (sum_i x_ij) / n, summed in FP64.
 *   centroid_dev [d] f64 out.
 * ------------------------------------------------------------------------- */
nsg_status nsg_centroid(const float *base_dev, int64_t n, int32_t d, double *centroid_dev,
                        void *stream);

/* ---------------------------------------------------------------------------
 * A3. Navigating node (Alg. 2; Section 3.5 step ii): Alg. 1 on the
 *   kNN graph from `start`, query = centroid, pool L; the navigating node is
 *   the first pool entry.  Distances to the centroid are FP64, summed over j
 *   in order without FMA contraction.  knn_ids_dev [n][K].
 *   Synchronises the stream; *nav_host receives the node.
 * ------------------------------------------------------------------------- */
nsg_status nsg_navigate(const float *base_dev, int64_t n, int32_t d, const int32_t *knn_ids_dev,
                        int32_t K, const double *centroid_dev, int32_t start, int32_t L,
                        int32_t *nav_host, void *stream);

/* ---------------------------------------------------------------------------
 * nsg_navigate_noalloc: nsg_navigate without any device allocation.  The
 *   paper has no counterpart; it exists for callers that may not allocate
 *   device memory themselves (a framework's caching allocator owns HBM, or a
 *   serving loop cannot afford cudaFree's device-wide synchronisation).
 *   Same arguments, result and synchronisation as nsg_navigate.  Its visited
 *   bitmap is a fixed array inside the library (held by every GPU that loads
 *   it until the process exits), so n <= NSG_NOALLOC_MAX_N, else NSG_EINVAL.
 *   The first call on a device looks the array up (cudaGetSymbolAddress); make
 *   that first call before any stream capture.  All calls on a device share
 *   the array (each clears what it uses first): calls that overlap on the GPU
 *   race and must be serialised by the caller.
 * ------------------------------------------------------------------------- */
#define NSG_NOALLOC_MAX_N 16777216
nsg_status nsg_navigate_noalloc(const float *base_dev, int64_t n, int32_t d, const int32_t *knn_ids_dev,
                                int32_t K, const double *centroid_dev, int32_t start, int32_t L,
                                int32_t *nav_host, void *stream);

/* ---------------------------------------------------------------------------
 * A5. Search-and-collect (Alg. 2; Section 3.5 step iii; Fig. 5) for
 *   nodes v0 .. v0+nv-1: Alg. 1 on the kNN graph from `nav` with query x_v
 *   and pool L; every node whose distance was computed, plus v's K kNN
 *   neighbours, minus v itself, sorted by key and cut to the C smallest.
 *   base_dev [n][d] with d % 4 == 0 and 16-byte aligned rows.
 *   cand_ids_dev [nv][C] i32, cand_d2_dev [nv][C] f32, cand_count_dev [nv]
 *   i32 out (row j describes node v0 + j).  status_dev [nv] i32 nullable.
 * ------------------------------------------------------------------------- */
nsg_status nsg_collect(const float *base_dev, int64_t n, int32_t d, const int32_t *knn_ids_dev,
                       int32_t K, int32_t nav, int32_t L, int32_t C, int64_t v0, int64_t nv,
                       int32_t *cand_ids_dev, float *cand_d2_dev, int32_t *cand_count_dev,
                       int32_t *status_dev, void *stream);

/* ---------------------------------------------------------------------------
 * A6. MRNG edge selection (Alg. 2; Def. MRNG and Section 3.3) for
 *   nodes v0 .. v0+nv-1 over their sorted candidates: the first candidate is
 *   kept; a later candidate p is dropped when some kept r has
 *   d2(p, r) < d2(p, v); stop at R kept.  Inputs as written by nsg_collect
 *   (a node's list ends at its count or at its first negative id).
 *   adj_dev [n][R] i32 and deg_dev [n] i32: rows v0.. are written (-1 padded).
 * ------------------------------------------------------------------------- */
nsg_status nsg_prune(const float *base_dev, int64_t n, int32_t d, const int32_t *cand_ids_dev,
                     const float *cand_d2_dev, const int32_t *cand_count_dev, int32_t C, int32_t R,
                     int64_t v0, int64_t nv, int32_t *adj_dev, int32_t *deg_dev, void *stream);

/* ---------------------------------------------------------------------------
 * A7. Connectivity (Alg. 2; Section 3.5 step iv): reach from
 *   `nav` (BFS; the same reached set as the paper's DFS tree).  While a node
 *   is unreached: u = smallest unreached id; Alg. 1 on the current graph from
 *   nav with query x_u and pool L; the first result (key order) whose
 *   out-degree is below R gets the edge s->u appended (else the smallest
 *   reached id with room; else NSG_EDEGREE); then everything reachable from
 *   u is marked.  adj_dev / deg_dev are updated in place.
 *   Synchronises the stream; *n_added_host receives the number of edges.
 * ------------------------------------------------------------------------- */
nsg_status nsg_connect(const float *base_dev, int64_t n, int32_t d, int32_t *adj_dev,
                       int32_t *deg_dev, int32_t R, int32_t nav, int32_t L, int32_t *n_added_host,
                       void *stream);

/* ---------------------------------------------------------------------------
 * Whole Alg. 2: A1 (K) -> A2 -> A3 (start = splitmix64(seed) mod n, pool L)
 *   -> A5/A6 for every node (L, C, R) -> A7 (L).  The base is copied into the
 *   index (the caller may free base_dev afterwards).  Requires 1 <= K < n,
 *   1 <= R <= C.  Synchronises the stream.
 * ------------------------------------------------------------------------- */
nsg_status nsg_build(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                     int32_t C, uint64_t seed, void *stream, nsg_index **out);

/* NSG-Naive (Section 4.1.2; the paper's ablation baseline): the MRNG edge
 *   selection applied directly to each node's K nearest neighbours (A1 then
 *   A6), with no navigating node and no connectivity pass.  The index's start
 *   node is splitmix64(seed) mod n; search it with params->init_random > 0
 *   for the paper's random initialisation.  K <= 256, R <= 1024.
 *   Synchronises the stream. */
nsg_status nsg_build_naive(const float *base_dev, int64_t n, int32_t d, int32_t K, int32_t R, uint64_t seed,
                           void *stream, nsg_index **out);

/* An index over a given graph (for searching a graph built elsewhere).
 *   adj_dev [n][R] (-1 padded; a row may list an id more than once, it is
 *   visited once), deg_dev [n] nullable (counted from adj when NULL).  Base
 *   and graph are copied. */
nsg_status nsg_index_from_graph(const float *base_dev, int64_t n, int32_t d, const int32_t *adj_dev,
                                const int32_t *deg_dev, int32_t R, int32_t nav, void *stream,
                                nsg_index **out);

/* ---------------------------------------------------------------------------
 * A4. Search on NSG (Alg. 1 started at the navigating node, Section 3.6), one
 *   warp per query: pool of L keys, expand the first unchecked entry, add its
 *   unvisited out-neighbours, keep the L smallest keys, stop when every entry
 *   is checked; return the first k.  queries_dev [nq][d] f32; ids_dev [nq][k]
 *   i32 out; d2_dev [nq][k] f32 out (nullable).  1 <= k <= L <= 1024.
 *   Returns NSG_ESTEPCAP (after the stream finishes) if any query hit its
 *   cap -- nsg_search synchronises only in that check.
 *   Warps draw queries from a device counter owned by the index (256 of
 *   them, used in turn): calls on one stream are ordered; at most 256 calls
 *   on one index may be in flight on different streams at once.  Batches
 *   larger than the GPU holds at once draw the queries farthest from the
 *   navigating node first (a launch ends with its last searches, and those
 *   tend to be the short ones then); each
 *   query's result does not depend on the order.  The order's scratch
 *   (12 bytes per query) comes from a stream-ordered memory pool the library
 *   keeps per device; when it cannot be had the batch runs in its own order.
 * nsg_search_ex: same with parameters and optional per-query outputs
 *   n_expand_dev [nq] (nodes checked), n_dist_dev [nq] (distances computed),
 *   status_dev [nq] (0, NSG_ESTEPCAP, or NSG_ECUDA for a staged copy that
 *   never landed, see stage_rows).  Does not synchronise.
 *   params->precision BF16 / FP8 (after nsg_index_prepare): traversal
 *   distances on that copy with FP32 accumulation; with re-rank, the L pool
 *   entries are measured again on the FP32 rows and the k smallest returned
 *   (d2 then holds FP32 squared distances; without re-rank, FP8 and lossy U8
 *   distances are in scaled units).  NSG_PREC_U8 sums squared byte
 *   differences exactly in int32 (__vabsdiffu4 + __dp4a); the query takes the
 *   copy's 8-bit map.
 * ------------------------------------------------------------------------- */
nsg_status nsg_search(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k,
                      int32_t L, int32_t *ids_dev, float *d2_dev, void *stream);
nsg_status nsg_search_ex(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k,
                         int32_t L, const nsg_search_params *params, int32_t *ids_dev,
                         float *d2_dev, int32_t *n_expand_dev, int32_t *n_dist_dev,
                         int32_t *status_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Partition-and-merge (Section 4.2, the NSG-16core experiment: random
 *   subsets, one NSG each, every query searched on every subset, results
 *   merged; Section 4.3: the same split across machines).
 * nsg_build_partitioned: part_host [n] i32 (HOST) gives each base row its
 *   subset 0..P-1; every subset needs >= 2 rows.  Subset p's rows, in
 *   ascending row order, get their own Alg. 2 build (kNN degree
 *   min(K, |subset| - 1), the same L, R, C and seed), ids local to it.  The
 *   index holds all subsets' graphs side by side in one allocation (subset p
 *   at positions off_p .. off_{p+1}-1, its navigating node off_p + nav_p),
 *   with the map from position to row id.  nsg_search / nsg_search_ex on it
 *   search subset 0 only and return positions; nsg_save refuses it.  The
 *   build phase times in nsg_index_info are sums over the subsets.
 *   Synchronises the stream.
 * nsg_search_partitioned: every query runs Alg. 1 on every subset's graph
 *   with pool L (one launch over nq x P (query, subset) units), then one
 *   warp per query merges the P result lists: the k smallest (distance, row
 *   id) keys of their union, ids as ROW ids.  ids_dev [nq][k] i32 out,
 *   d2_dev [nq][k] f32 out (nullable), -1 / +inf padded when the subsets
 *   hold fewer than k rows in all.  params as nsg_search_ex, without the
 *   learned stop or random initialisation (NSG_EINVAL).  Per-unit results
 *   go to scratch owned by the index (grown on demand, so a larger batch
 *   than any before allocates and synchronises once); calls on one index on
 *   different streams at once race on it.  Asynchronous otherwise.
 * ------------------------------------------------------------------------- */
nsg_status nsg_build_partitioned(const float *base_dev, int64_t n, int32_t d, const int32_t *part_host,
                                 int32_t P, int32_t K, int32_t L, int32_t R, int32_t C, uint64_t seed,
                                 void *stream, nsg_index **out);
nsg_status nsg_search_partitioned(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k,
                                  int32_t L, const nsg_search_params *params, int32_t *ids_dev, float *d2_dev,
                                  void *stream);

/* ---------------------------------------------------------------------------
 * nsg_search_host: nsg_search_ex on HOST buffers (not in the paper: the
 *   serving-side call).  queries_host [nq][d] f32 in, ids_host [nq][k] i32
 *   out, d2_host [nq][k] f32 out (nullable); page-locked host memory copies
 *   fastest, pageable memory works.  On `stream`: one host->device copy of
 *   the queries into device staging owned by the index (grown on demand,
 *   kept until nsg_free), one search launch over the whole batch, the
 *   device->host copies of the results.  Calls on one index are serialised.
 *   Synchronous: returns once the results are in host memory (on an error,
 *   after the stream has drained), with NSG_ESTEPCAP if any query hit its
 *   step cap (its partial result is kept).
 * ------------------------------------------------------------------------- */
nsg_status nsg_search_host(const nsg_index *idx, const float *queries_host, int64_t nq, int32_t k,
                           int32_t L, const nsg_search_params *params, int32_t *ids_host,
                           float *d2_host, void *stream);

/* ---------------------------------------------------------------------------
 * Batched uneven queries (not in the paper: a serving-side addition).  Query
 *   q asks for k_dev[q] results with pool L_dev[q] (clamped to 1..kmax and
 *   max(k_q, .)..Lmax).  Outputs are [nq][kmax] rows, padded with -1 / +inf
 *   past each query's k.  One persistent launch: warps draw queries from a
 *   device work counter, longest pool first.
 * nsg_search_batched: one-shot form (derives the visiting order each call).
 * nsg_plan_create: binds an index, the query / k / L / output buffers and
 *   the parameters; derives the visiting order; with `autotune` times the
 *   candidate launch shapes (pool placement shared / global memory -- global
 *   only when Lmax > 1024, or fixed by params->pool -- x warps per query
 *   1/2/4 x warps per block 2/4/8 x visited-hash slots 512/1024/2048; shapes
 *   with fewer warps per block than per query skipped, 24 per placement) on
 *   the bound batch and keeps the fastest;
 *   then captures
 *   "reset work counter + search" as a CUDA graph.  Synchronises.
 * nsg_plan_run: replays the graph on `stream` (asynchronous).
 * nsg_plan_info: the chosen shape and the tuning timings.
 * ------------------------------------------------------------------------- */
typedef struct nsg_plan nsg_plan;
typedef struct {
    int32_t warps_per_cta; /* chosen launch shape */
    int32_t hash_slots;
    int32_t n_tried;       /* shapes timed by the autotuner (0: none) */
    float best_ms;         /* time of one run of the chosen shape (autotune only) */
    float worst_ms;        /* slowest shape tried */
    int32_t warps_per_query; /* chosen warps per query */
    int32_t pool;          /* chosen pool placement: 1 shared memory, 2 global memory */
    int32_t stage_rows;    /* chosen staged-gather slots per warp (0: register gathers) */
} nsg_plan_info_t;

nsg_status nsg_search_batched(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                              const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                              int32_t *ids_dev, float *d2_dev, int32_t *status_dev, void *stream);
nsg_status nsg_plan_create(const nsg_index *idx, const float *queries_dev, int64_t nq, const int32_t *k_dev,
                           const int32_t *L_dev, int32_t kmax, int32_t Lmax, const nsg_search_params *params,
                           int32_t *ids_dev, float *d2_dev, int32_t *status_dev, int32_t autotune, void *stream,
                           nsg_plan **out);
nsg_status nsg_plan_run(nsg_plan *plan, void *stream);
nsg_status nsg_plan_info(const nsg_plan *plan, nsg_plan_info_t *info);
void nsg_plan_free(nsg_plan *plan);

/* ---------------------------------------------------------------------------
 * Learned early termination (not in the paper: a serving-side addition; the
 * fixed-L Alg. 1 is its fallback and the yardstick of its recall loss).
 * nsg_search_trace: Alg. 1 with fixed L that records, before each expansion
 *   t (t < cap), the 8 state features (feat_dev [nq][cap][8] f32) and after
 *   it whether the first stop_k pool entries changed (flag_dev [nq][cap] u8);
 *   steps_dev [nq] receives the expansion count.  params as nsg_search_ex
 *   (stop_model ignored).  ids_dev [nq][k] receives the results.
 * nsg_stop_train: full-batch Adam on those traces; the label of step t is 1
 *   when no later step changes the first stop_k entries.  master_dev: FP32
 *   parameters [NSG_STOP_PARAMS] (initialised from `seed` when seed != 0,
 *   else continued); model_dev: FP16 export [NSG_STOP_PARAMS] for
 *   params->stop_model; loss_dev [iters] (nullable): mean BCE per iteration.
 *   Synchronises the stream.
 * ------------------------------------------------------------------------- */
nsg_status nsg_search_trace(const nsg_index *idx, const float *queries_dev, int64_t nq, int32_t k, int32_t L,
                            const nsg_search_params *params, int32_t *ids_dev, float *feat_dev,
                            uint8_t *flag_dev, int32_t *steps_dev, int32_t cap, void *stream);
nsg_status nsg_stop_train(const float *feat_dev, const uint8_t *flag_dev, const int32_t *steps_dev, int64_t nq,
                          int32_t cap, int32_t iters, float lr, uint64_t seed, float *master_dev, void *model_dev,
                          float *loss_dev, void *stream);

/* ---------------------------------------------------------------------------
 * A8. Precision (Eq. 1): hits_dev[q] = |{first k of ids} n {first k of gt}|.
 *   ids_dev [nq][ld_ids], gt_dev [nq][ld_gt], hits_dev [nq] i32 out.
 * ------------------------------------------------------------------------- */
nsg_status nsg_recall(const int32_t *ids_dev, int32_t ld_ids, const int32_t *gt_dev, int32_t ld_gt,
                      int64_t nq, int32_t k, int32_t *hits_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Index management.
 * nsg_index_info: sizes, navigating node, degree statistics, build times.
 * nsg_index_graph: copy the adjacency [n][R] and degrees [n] to device
 *   buffers (either nullable); async on stream.
 * nsg_save / nsg_load: little-endian file: magic "NSGGB300", version, n, d,
 *   R, nav, then deg [n] i32, adj [n][R] i32, base [n][d] f32.  Synchronous.
 * nsg_free: releases the index (NULL is ignored).
 * ------------------------------------------------------------------------- */
nsg_status nsg_index_info(const nsg_index *idx, nsg_index_info_t *info);
/* Low-precision copy of the base for the precision forms of nsg_search_ex
 *   (NSG_PREC_BF16: round to nearest; NSG_PREC_FP8: e4m3 of x * s with
 *   s = 448 / max|x|, saturating; NSG_PREC_U8: rint((x - lo) * s) with
 *   lo = min x and s = 1 when every value is an integer and max - min <= 255,
 *   else s = 255 / (max - min)).  Owned by the index; a no-op when present.
 *   Synchronises the stream. */
nsg_status nsg_index_prepare(nsg_index *idx, int32_t precision, void *stream);
nsg_status nsg_index_graph(const nsg_index *idx, int32_t *adj_dev, int32_t *deg_dev, void *stream);
nsg_status nsg_save(const nsg_index *idx, const char *path);
nsg_status nsg_load(const char *path, void *stream, nsg_index **out);
void nsg_free(nsg_index *idx);

#ifdef __cplusplus
}
#endif
#endif /* NSG_H */
