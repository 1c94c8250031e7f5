/*
 * nsg_oracle.c -- plain, slow, obviously-correct CPU oracle for the hot path of
 * the Navigating Spreading-out Graph (Fu, Xiang, Wang, Cai: "Fast Approximate
 * Nearest Neighbor Search With The Navigating Spreading-out Graph").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Everything runs in the order the paper states it:
 *   - distance: squared l2 (Section 2: delta is the l2 distance; squaring keeps
 *     every comparison), accumulated in float over j = 0..d-1, no FMA
 *     contraction (built with -ffp-contract=off);
 *   - key order: (dist, id) ascending everywhere (Alg. 1 sorts by distance;
 *     the lower index breaks isosceles ties in the MRNG definition, Sec. 3.3);
 *   - Alg. 1 (Search-on-Graph), Alg. 2 (NSGbuild) with its centroid, navigating
 *     node, search-and-collect, MRNG edge selection and DFS-tree connectivity;
 *   - the naive MRNG construction of Section 3.4 and exact kNN by serial scan
 *     (Section 4.1.2, item 1).
 * Threads (pthreads) only split loops over independent queries / nodes /
 * column ranges whose results are merged by key, so every output is identical
 * for any thread count.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   R1  Alg. 1 loop: "while i < l" never ends when |S| < l and every entry is
 *       checked; the loop stops when no unchecked entry is left.
 *   R2  S is a set: a node whose distance was computed once is never added
 *       again (identical to re-adding, see the proof in the design notes).
 *   R3  search-and-collect keeps every *visited* node (distance computed;
 *       Sec. 3.5 step iii-(2) and Fig. 5), plus all K kNN neighbours of v, minus
 *       v itself; sorted by key and cut to the C smallest (C is a build cap).
 *   R4  edge selection: p is occluded when some kept r has dist(p,r) <
 *       dist(p,v) (r in the open lune of vp; Def. MRNG and Sec. 3.3); the first
 *       candidate is always kept; stop at m = R kept.
 *   R5  random start node r = splitmix64(seed) mod n.
 *   R6  the navigating-node search measures distances to the centroid in
 *       double, sum over j in order, no FMA.
 *   R7  connectivity: BFS reach from the navigating node (same reached set as
 *       DFS); u = smallest unreached id; Alg. 1 on the current graph from the
 *       navigating node with query x_u; the first result (key order) with
 *       out-degree < R gets the edge s->u; else the smallest reached id with
 *       out-degree < R; else error.  Then everything reachable from u is
 *       marked.
 *   R10 NSG-Naive's "Alg. 1 with random initialization": the pool starts as
 *       the set of `count` seeded random nodes (count <= L), query q drawing
 *       splitmix64(seed + q * 0x9e3779b97f4a7c15 + j) mod n for j < count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EDEGREE -5

/* ------------------------------------------------------------------------ */
/* distance and key order                                                    */
/* ------------------------------------------------------------------------ */

/* Squared l2 distance, float, summed over j = 0..d-1 (Section 2). */
float orc_dist2(const float *a, const float *b, int32_t d) {
    float s = 0.0f;
    for (int32_t j = 0; j < d; ++j) {
        float t = a[j] - b[j];
        s = s + t * t;
    }
    return s;
}

/* Squared l2 distance to a double-precision point (reading R6). */
static double dist2_f64(const float *a, const double *c, int32_t d) {
    double s = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        double t = (double)a[j] - c[j];
        s = s + t * t;
    }
    return s;
}

typedef struct {
    double dist; /* float distances are widened exactly */
    int32_t id;
    int32_t checked;
} entry;

static int entry_cmp(const void *pa, const void *pb) {
    const entry *a = (const entry *)pa, *b = (const entry *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* ------------------------------------------------------------------------ */
/* tiny thread pool: run fn(i) for i in [0, count) split over nthreads        */
/* ------------------------------------------------------------------------ */

typedef void (*unit_fn)(void *ctx, int64_t i);
typedef struct {
    unit_fn fn;
    void *ctx;
    int64_t lo, hi;
} span_arg;

static void *span_run(void *p) {
    span_arg *a = (span_arg *)p;
    for (int64_t i = a->lo; i < a->hi; ++i) a->fn(a->ctx, i);
    return NULL;
}

static void run_units(unit_fn fn, void *ctx, int64_t count, int32_t nthreads) {
    if (nthreads <= 1 || count <= 1) {
        for (int64_t i = 0; i < count; ++i) fn(ctx, i);
        return;
    }
    if (nthreads > count) nthreads = (int32_t)count;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    span_arg *args = (span_arg *)malloc(sizeof(span_arg) * nthreads);
    for (int32_t t = 0; t < nthreads; ++t) {
        args[t].fn = fn;
        args[t].ctx = ctx;
        args[t].lo = count * t / nthreads;
        args[t].hi = count * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, span_run, &args[t]);
    }
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
}

/* ------------------------------------------------------------------------ */
/* exact k nearest neighbours by serial scan (Section 4.1.2 item 1)          */
/* ------------------------------------------------------------------------ */

/* Insert (dist,id) into a sorted list of at most k entries. */
static void topk_push(entry *list, int32_t *size, int32_t k, double dist, int32_t id) {
    entry e = {dist, id, 0};
    if (*size == k && entry_cmp(&e, &list[k - 1]) >= 0) return;
    int32_t pos = (*size < k) ? *size : k - 1;
    while (pos > 0 && entry_cmp(&e, &list[pos - 1]) < 0) {
        list[pos] = list[pos - 1];
        --pos;
    }
    list[pos] = e;
    if (*size < k) ++*size;
}

/* Scan base rows [lo, hi) for the k nearest to q (skipping id `skip`). */
static int32_t scan_range(const float *base, int32_t d, const float *q, int64_t lo, int64_t hi,
                          int64_t skip, int32_t k, entry *list) {
    int32_t size = 0;
    for (int64_t j = lo; j < hi; ++j) {
        if (j == skip) continue;
        topk_push(list, &size, k, (double)orc_dist2(q, base + j * d, d), (int32_t)j);
    }
    return size;
}

typedef struct {
    const float *base;
    int64_t n;
    int32_t d, k;
    const float *q;
    int64_t skip;
    int32_t nparts;
    entry *lists; /* [nparts][k] */
    int32_t *sizes;
} scan_ctx;

static void scan_part(void *p, int64_t t) {
    scan_ctx *c = (scan_ctx *)p;
    int64_t lo = c->n * t / c->nparts, hi = c->n * (t + 1) / c->nparts;
    c->sizes[t] = scan_range(c->base, c->d, c->q, lo, hi, c->skip, c->k, c->lists + t * c->k);
}

/* One query, column range split over threads, partial lists merged by key. */
static int knn_one(const float *base, int64_t n, int32_t d, const float *q, int64_t skip, int32_t k,
                   int32_t nthreads, int32_t *ids, float *dist) {
    int32_t parts = nthreads < 1 ? 1 : nthreads;
    scan_ctx c = {base, n, d, k, q, skip, parts, NULL, NULL};
    c.lists = (entry *)malloc(sizeof(entry) * (size_t)parts * k);
    c.sizes = (int32_t *)calloc(parts, sizeof(int32_t));
    entry *merged = (entry *)malloc(sizeof(entry) * k);
    if (!c.lists || !c.sizes || !merged) return ORC_ENOMEM;
    run_units(scan_part, &c, parts, parts);
    int32_t size = 0;
    for (int32_t t = 0; t < parts; ++t)
        for (int32_t i = 0; i < c.sizes[t]; ++i)
            topk_push(merged, &size, k, c.lists[t * k + i].dist, c.lists[t * k + i].id);
    for (int32_t i = 0; i < k; ++i) {
        ids[i] = i < size ? merged[i].id : -1;
        if (dist) dist[i] = i < size ? (float)merged[i].dist : INFINITY;
    }
    free(c.lists);
    free(c.sizes);
    free(merged);
    return ORC_OK;
}

typedef struct {
    const float *base, *qry;
    int64_t n;
    int32_t d, k, self;
    const int64_t *rows;
    int32_t *ids;
    float *dist;
} knn_ctx;

static void knn_unit(void *p, int64_t i) {
    knn_ctx *c = (knn_ctx *)p;
    int64_t row = c->rows ? c->rows[i] : i;
    const float *q = c->self ? c->base + row * c->d : c->qry + i * c->d;
    knn_one(c->base, c->n, c->d, q, c->self ? row : -1, c->k, 1, c->ids + i * c->k,
            c->dist ? c->dist + i * c->k : NULL);
}

/* kNN graph rows: for each listed base row (all rows when rows == NULL), the k
 * nearest other base rows by key; self excluded by id (Alg. 2 input G). */
int orc_knn_rows(const float *base, int64_t n, int32_t d, int32_t k, const int64_t *rows,
                 int64_t nrows, int32_t nthreads, int32_t *ids, float *dist) {
    if (!base || !ids || n < 1 || d < 1 || k < 1) return ORC_EINVAL;
    knn_ctx c = {base, NULL, n, d, k, 1, rows, ids, dist};
    if (nrows < nthreads && nthreads > 1) {
        for (int64_t i = 0; i < nrows; ++i) {
            int64_t row = rows ? rows[i] : i;
            int rc = knn_one(base, n, d, base + row * d, row, k, nthreads, ids + i * k,
                             dist ? dist + i * k : NULL);
            if (rc) return rc;
        }
        return ORC_OK;
    }
    run_units(knn_unit, &c, rows ? nrows : n, nthreads);
    return ORC_OK;
}

/* Exact k nearest base rows for each query (ground truth, serial scan). */
int orc_knn_query(const float *base, int64_t n, int32_t d, const float *qry, int64_t nq, int32_t k,
                  int32_t nthreads, int32_t *ids, float *dist) {
    if (!base || !qry || !ids || n < 1 || d < 1 || k < 1) return ORC_EINVAL;
    knn_ctx c = {base, qry, n, d, k, 0, NULL, ids, dist};
    run_units(knn_unit, &c, nq, nthreads);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* graphs: fixed-width adjacency, or a kNN graph whose rows are computed on  */
/* first use (lets the oracle follow a search on a large base row by row)    */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* fixed-width adjacency [n][width], -1 padded; deg may be NULL */
    const int32_t *adj;
    const int32_t *deg;
    int32_t width;
    /* lazy kNN graph (adj == NULL) */
    struct orc_lazy_knn *lazy;
} graph;

struct orc_lazy_knn {
    const float *base;
    int64_t n;
    int32_t d, k, nthreads;
    int32_t *ids;  /* [n][k] */
    uint8_t *have; /* [n] */
    int64_t rows_computed;
};

typedef struct orc_lazy_knn orc_lazy_knn;

orc_lazy_knn *orc_lazy_knn_new(const float *base, int64_t n, int32_t d, int32_t k,
                               int32_t nthreads) {
    orc_lazy_knn *g = (orc_lazy_knn *)calloc(1, sizeof(orc_lazy_knn));
    g->base = base;
    g->n = n;
    g->d = d;
    g->k = k;
    g->nthreads = nthreads;
    g->ids = (int32_t *)calloc((size_t)n * k, sizeof(int32_t));
    g->have = (uint8_t *)calloc((size_t)n, 1);
    return g;
}

void orc_lazy_knn_free(orc_lazy_knn *g) {
    if (!g) return;
    free(g->ids);
    free(g->have);
    free(g);
}

const int32_t *orc_lazy_knn_row(orc_lazy_knn *g, int32_t u) {
    if (!g->have[u]) {
        knn_one(g->base, g->n, g->d, g->base + (int64_t)u * g->d, u, g->k, g->nthreads,
                g->ids + (int64_t)u * g->k, NULL);
        g->have[u] = 1;
        g->rows_computed++;
    }
    return g->ids + (int64_t)u * g->k;
}

int64_t orc_lazy_knn_rows_computed(const orc_lazy_knn *g) { return g->rows_computed; }

static int32_t graph_row(const graph *g, int32_t u, const int32_t **row) {
    if (g->lazy) {
        *row = orc_lazy_knn_row(g->lazy, u);
        return g->lazy->k;
    }
    *row = g->adj + (int64_t)u * g->width;
    if (g->deg) return g->deg[u];
    int32_t c = 0;
    while (c < g->width && (*row)[c] >= 0) ++c;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1  Search-on-Graph(G, p, q, l)                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    const float *base;
    int32_t d;
    const float *q;    /* float query, or */
    const double *qd;  /* double query (navigating-node search, reading R6) */
} metric;

static double metric_dist(const metric *m, int32_t id) {
    const float *x = m->base + (int64_t)id * m->d;
    if (m->qd) return dist2_f64(x, m->qd, m->d);
    return (double)orc_dist2(m->q, x, m->d);
}

typedef struct {
    entry *items;
    int64_t size, cap;
} entry_vec;

static void vec_push(entry_vec *v, double dist, int32_t id) {
    if (v->size == v->cap) {
        v->cap = v->cap ? v->cap * 2 : 256;
        v->items = (entry *)realloc(v->items, sizeof(entry) * v->cap);
    }
    v->items[v->size].dist = dist;
    v->items[v->size].id = id;
    v->items[v->size].checked = 0;
    v->size++;
}

/*
 * Alg. 1 from start node p with pool size l.  S (capacity l + max degree) holds
 * the pool on return, sorted by key; returns |S|.  `visited` (n bytes, zero on
 * entry) marks every node whose distance was computed.  When `seen` is given,
 * every visited (dist, id) is appended to it (search-and-collect).  When
 * `trace` is given, the ids of S after each expansion are written to
 * trace[step][0..l) (-1 padded) for up to trace_steps steps.
 */
static int32_t alg1_from(const graph *g, const metric *m, const int32_t *init, int32_t n_init,
                         int32_t l, entry *S, uint8_t *visited, entry_vec *seen, int32_t *trace,
                         int32_t trace_steps, int64_t *n_expand, int64_t *n_dist) {
    /* S starts as the set of the given nodes (duplicates once), sorted by key */
    int32_t size = 0;
    for (int32_t t = 0; t < n_init; ++t) {
        int32_t p = init[t];
        if (visited[p]) continue;
        visited[p] = 1;
        double dp = metric_dist(m, p);
        *n_dist += 1;
        if (seen) vec_push(seen, dp, p);
        S[size].dist = dp;
        S[size].id = p;
        S[size].checked = 0;
        size++;
    }
    qsort(S, size, sizeof(entry), entry_cmp);
    if (size > l) size = l;
    int64_t step = 0;
    for (;;) {
        int32_t i = 0;
        while (i < size && S[i].checked) ++i; /* first unchecked node in S */
        if (i == size) break;                  /* reading R1 */
        S[i].checked = 1;
        *n_expand += 1;
        const int32_t *nb;
        int32_t cnt = graph_row(g, S[i].id, &nb);
        for (int32_t t = 0; t < cnt; ++t) {
            int32_t v = nb[t];
            if (v < 0 || visited[v]) continue; /* reading R2 */
            visited[v] = 1;
            double dv = metric_dist(m, v);
            *n_dist += 1;
            if (seen) vec_push(seen, dv, v);
            S[size].dist = dv;
            S[size].id = v;
            S[size].checked = 0;
            size++;
        }
        qsort(S, size, sizeof(entry), entry_cmp); /* sort S by distance to q */
        if (size > l) size = l;                   /* resize to l */
        if (trace && step < trace_steps) {
            for (int32_t t = 0; t < l; ++t) trace[step * l + t] = t < size ? S[t].id : -1;
        }
        step++;
    }
    return size;
}

static int32_t alg1(const graph *g, const metric *m, int32_t p, int32_t l, entry *S,
                    uint8_t *visited, entry_vec *seen, int32_t *trace, int32_t trace_steps,
                    int64_t *n_expand, int64_t *n_dist) {
    return alg1_from(g, m, &p, 1, l, S, visited, seen, trace, trace_steps, n_expand, n_dist);
}

static int32_t graph_max_width(const graph *g) { return g->lazy ? g->lazy->k : g->width; }

/* Search on a fixed graph (Alg. 1, Section 3.6): for each query, start at
 * `start`, pool size l, return the first k ids (-1 / +inf padded). */
typedef struct {
    graph g;
    const float *base, *qry;
    int64_t n;
    int32_t d, start, l, k;
    int32_t *ids;
    float *dist;
    int64_t *n_expand, *n_dist;
} search_ctx;

static void search_unit(void *p, int64_t qi) {
    search_ctx *c = (search_ctx *)p;
    entry *S = (entry *)malloc(sizeof(entry) * (c->l + graph_max_width(&c->g) + 1));
    uint8_t *visited = (uint8_t *)calloc((size_t)c->n, 1);
    metric m = {c->base, c->d, c->qry + qi * c->d, NULL};
    int64_t ne = 0, nd = 0;
    int32_t size = alg1(&c->g, &m, c->start, c->l, S, visited, NULL, NULL, 0, &ne, &nd);
    for (int32_t t = 0; t < c->k; ++t) {
        c->ids[qi * c->k + t] = t < size ? S[t].id : -1;
        if (c->dist) c->dist[qi * c->k + t] = t < size ? (float)S[t].dist : INFINITY;
    }
    if (c->n_expand) c->n_expand[qi] = ne;
    if (c->n_dist) c->n_dist[qi] = nd;
    free(S);
    free(visited);
}

int orc_search(const int32_t *adj, const int32_t *deg, int64_t n, int32_t width, const float *base,
               int32_t d, int32_t start, const float *qry, int64_t nq, int32_t k, int32_t l,
               int32_t nthreads, int32_t *ids, float *dist, int64_t *n_expand, int64_t *n_dist) {
    if (!adj || !base || !qry || !ids || n < 1 || d < 1 || k < 1 || l < 1 || start < 0 ||
        start >= n)
        return ORC_EINVAL;
    search_ctx c = {{adj, deg, width, NULL}, base, qry, n, d, start, l, k, ids, dist, n_expand, n_dist};
    run_units(search_unit, &c, nq, nthreads);
    return ORC_OK;
}

/* Alg. 1 with random initialisation (NSG-Naive, Section 4.1.2; reading R10):
 * query qi's pool starts as the set of nodes
 *   splitmix64(seed + qi * 0x9e3779b97f4a7c15 + j) mod n,  j = 0 .. count-1
 * (repeats once), then Alg. 1 runs as usual. */
uint64_t orc_splitmix64(uint64_t x);

typedef struct {
    search_ctx s;
    int32_t count;
    uint64_t seed;
} search_rand_ctx;

static void search_rand_unit(void *p, int64_t qi) {
    search_rand_ctx *c = (search_rand_ctx *)p;
    entry *S = (entry *)malloc(sizeof(entry) * (c->s.l + c->count + graph_max_width(&c->s.g) + 1));
    uint8_t *visited = (uint8_t *)calloc((size_t)c->s.n, 1);
    int32_t *init = (int32_t *)malloc(sizeof(int32_t) * c->count);
    for (int32_t j = 0; j < c->count; ++j)
        init[j] = (int32_t)(orc_splitmix64(c->seed + (uint64_t)qi * 0x9e3779b97f4a7c15ULL + (uint64_t)j) %
                            (uint64_t)c->s.n);
    metric m = {c->s.base, c->s.d, c->s.qry + qi * c->s.d, NULL};
    int64_t ne = 0, nd = 0;
    int32_t size = alg1_from(&c->s.g, &m, init, c->count, c->s.l, S, visited, NULL, NULL, 0, &ne, &nd);
    for (int32_t t = 0; t < c->s.k; ++t) {
        c->s.ids[qi * c->s.k + t] = t < size ? S[t].id : -1;
        if (c->s.dist) c->s.dist[qi * c->s.k + t] = t < size ? (float)S[t].dist : INFINITY;
    }
    if (c->s.n_expand) c->s.n_expand[qi] = ne;
    if (c->s.n_dist) c->s.n_dist[qi] = nd;
    free(init);
    free(S);
    free(visited);
}

int orc_search_random(const int32_t *adj, const int32_t *deg, int64_t n, int32_t width,
                      const float *base, int32_t d, const float *qry, int64_t nq, int32_t k, int32_t l,
                      int32_t count, uint64_t seed, int32_t nthreads, int32_t *ids, float *dist,
                      int64_t *n_expand, int64_t *n_dist) {
    if (!adj || !base || !qry || !ids || n < 1 || d < 1 || k < 1 || l < 1 || count < 1 || count > l)
        return ORC_EINVAL;
    search_rand_ctx c = {{{adj, deg, width, NULL}, base, qry, n, d, 0, l, k, ids, dist, n_expand, n_dist},
                         count, seed};
    run_units(search_rand_unit, &c, nq, nthreads);
    return ORC_OK;
}

/* One query with the pool after every expansion written to trace[step][l]. */
int orc_search_trace(const int32_t *adj, const int32_t *deg, int64_t n, int32_t width,
                     const float *base, int32_t d, int32_t start, const float *q, int32_t l,
                     int32_t *trace, int32_t trace_steps, int64_t *steps_out) {
    if (!adj || !base || !q || l < 1) return ORC_EINVAL;
    graph g = {adj, deg, width, NULL};
    entry *S = (entry *)malloc(sizeof(entry) * (l + width + 1));
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    metric m = {base, d, q, NULL};
    int64_t ne = 0, nd = 0;
    alg1(&g, &m, start, l, S, visited, NULL, trace, trace_steps, &ne, &nd);
    if (steps_out) *steps_out = ne;
    free(S);
    free(visited);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 NSGbuild(G, l, m)                                                  */
/* ------------------------------------------------------------------------ */

/* Published SplitMix64 finaliser (Steele, Lea, Flood 2014); reading R5. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Alg. 2, centroid step: the centroid, summed in double over i in order, then / n. */
int orc_centroid(const float *base, int64_t n, int32_t d, double *c) {
    if (!base || !c || n < 1 || d < 1) return ORC_EINVAL;
    for (int32_t j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s = s + (double)base[i * d + j];
        c[j] = s / (double)n;
    }
    return ORC_OK;
}

/* Alg. 2, navigating-node step: Alg. 1 on the kNN graph from r toward the centroid;
 * the navigating node is the nearest pool entry. */
static int32_t navigate(const graph *knn, const float *base, int64_t n, int32_t d,
                        const double *c, int32_t r, int32_t l) {
    entry *S = (entry *)malloc(sizeof(entry) * (l + graph_max_width(knn) + 1));
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    metric m = {base, d, NULL, c};
    int64_t ne = 0, nd = 0;
    alg1(knn, &m, r, l, S, visited, NULL, NULL, 0, &ne, &nd);
    int32_t nav = S[0].id;
    free(S);
    free(visited);
    return nav;
}

int orc_navigate(const int32_t *knn, int64_t n, int32_t K, const float *base, int32_t d,
                 const double *c, int32_t r, int32_t l, int32_t *nav) {
    if (!knn || !base || !c || !nav || r < 0 || r >= n) return ORC_EINVAL;
    graph g = {knn, NULL, K, NULL};
    *nav = navigate(&g, base, n, d, c, r, l);
    return ORC_OK;
}

int orc_navigate_lazy(orc_lazy_knn *knn, const double *c, int32_t r, int32_t l, int32_t *nav) {
    graph g = {NULL, NULL, 0, knn};
    *nav = navigate(&g, knn->base, knn->n, knn->d, c, r, l);
    return ORC_OK;
}

/* Alg. 2, search-and-collect step (reading R3): candidates of node v, sorted, cut to C.
 * Returns the count written to cand_ids / cand_dist. */
static int32_t collect(const graph *knn, const int32_t *knn_row_v, int32_t K, const float *base,
                       int64_t n, int32_t d, int32_t nav, int32_t v, int32_t l, int32_t C,
                       int32_t *cand_ids, float *cand_dist, int64_t *n_expand, int64_t *n_dist) {
    entry *S = (entry *)malloc(sizeof(entry) * (l + graph_max_width(knn) + 1));
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    entry_vec seen = {NULL, 0, 0};
    const float *q = base + (int64_t)v * d;
    metric m = {base, d, q, NULL};
    int64_t ne = 0, nd = 0;
    alg1(knn, &m, nav, l, S, visited, &seen, NULL, 0, &ne, &nd);
    for (int32_t t = 0; t < K; ++t) { /* add v's nearest neighbours in G */
        int32_t w = knn_row_v[t];
        if (w < 0 || visited[w]) continue;
        visited[w] = 1;
        vec_push(&seen, (double)orc_dist2(q, base + (int64_t)w * d, d), w);
    }
    int64_t kept = 0; /* drop v itself */
    for (int64_t t = 0; t < seen.size; ++t)
        if (seen.items[t].id != v) seen.items[kept++] = seen.items[t];
    qsort(seen.items, kept, sizeof(entry), entry_cmp);
    int32_t cnt = kept < C ? (int32_t)kept : C;
    for (int32_t t = 0; t < cnt; ++t) {
        cand_ids[t] = seen.items[t].id;
        cand_dist[t] = (float)seen.items[t].dist;
    }
    for (int32_t t = cnt; t < C; ++t) {
        cand_ids[t] = -1;
        cand_dist[t] = INFINITY;
    }
    if (n_expand) *n_expand = ne;
    if (n_dist) *n_dist = nd;
    free(seen.items);
    free(S);
    free(visited);
    return cnt;
}

/* Alg. 2, edge-selection loop (reading R4): MRNG edge selection over sorted candidates.
 * Writes up to R ids to out (-1 padded); returns the kept count. */
static int32_t mrng_select(const float *base, int32_t d, const int32_t *cand_ids,
                           const float *cand_dist, int32_t ncand, int32_t R, int32_t *out) {
    int32_t kept = 0;
    if (ncand > 0 && R > 0) out[kept++] = cand_ids[0];
    for (int32_t t = 1; t < ncand && kept < R; ++t) {
        int32_t p = cand_ids[t];
        const float *xp = base + (int64_t)p * d;
        int occluded = 0;
        for (int32_t s = 0; s < kept; ++s) {
            if (orc_dist2(xp, base + (int64_t)out[s] * d, d) < cand_dist[t]) {
                occluded = 1;
                break;
            }
        }
        if (!occluded) out[kept++] = p;
    }
    for (int32_t t = kept; t < R; ++t) out[t] = -1;
    return kept;
}

int orc_prune(const float *base, int32_t d, const int32_t *cand_ids, const float *cand_dist,
              int32_t ncand, int32_t R, int32_t *out, int32_t *deg) {
    if (!base || !out || R < 1) return ORC_EINVAL;
    int32_t k = mrng_select(base, d, cand_ids, cand_dist, ncand, R, out);
    if (deg) *deg = k;
    return ORC_OK;
}

/* Candidates for one node on a full kNN graph. */
int orc_collect(const int32_t *knn, int32_t K, const float *base, int64_t n, int32_t d,
                int32_t nav, int32_t v, int32_t l, int32_t C, int32_t *cand_ids, float *cand_dist,
                int32_t *count, int64_t *n_expand, int64_t *n_dist) {
    if (!knn || !base || !cand_ids || !cand_dist || v < 0 || v >= n) return ORC_EINVAL;
    graph g = {knn, NULL, K, NULL};
    int32_t c = collect(&g, knn + (int64_t)v * K, K, base, n, d, nav, v, l, C, cand_ids, cand_dist,
                        n_expand, n_dist);
    if (count) *count = c;
    return ORC_OK;
}

/* Candidates for one node on a lazily computed kNN graph (large n). */
int orc_collect_lazy(orc_lazy_knn *knn, int32_t nav, int32_t v, int32_t l, int32_t C,
                     int32_t *cand_ids, float *cand_dist, int32_t *count) {
    graph g = {NULL, NULL, 0, knn};
    const int32_t *row = orc_lazy_knn_row(knn, v);
    int32_t c = collect(&g, row, knn->k, knn->base, knn->n, knn->d, nav, v, l, C, cand_ids,
                        cand_dist, NULL, NULL);
    if (count) *count = c;
    return ORC_OK;
}

/* BFS over the fixed-width graph from `root`, marking unreached nodes. */
static void mark_reachable(const int32_t *adj, const int32_t *deg, int32_t R, int32_t root,
                           uint8_t *reached, int32_t *queue) {
    if (reached[root]) return;
    int64_t head = 0, tail = 0;
    reached[root] = 1;
    queue[tail++] = root;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t t = 0; t < deg[u]; ++t) {
            int32_t v = adj[(int64_t)u * R + t];
            if (v >= 0 && !reached[v]) {
                reached[v] = 1;
                queue[tail++] = v;
            }
        }
    }
}

/* Alg. 2, connectivity step (reading R7).  adj/deg are updated in place. */
int orc_connect(int32_t *adj, int32_t *deg, int64_t n, int32_t R, const float *base, int32_t d,
                int32_t nav, int32_t l, int32_t *n_added, int32_t *added, int32_t added_cap) {
    if (!adj || !deg || !base || nav < 0 || nav >= n) return ORC_EINVAL;
    uint8_t *reached = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    entry *S = (entry *)malloc(sizeof(entry) * (l + R + 1));
    uint8_t *visited = (uint8_t *)malloc((size_t)n);
    int rc = ORC_OK;
    int32_t count = 0;
    mark_reachable(adj, deg, R, nav, reached, queue);
    int64_t u = 0;
    for (;;) {
        while (u < n && reached[u]) ++u;
        if (u == n) break;
        memset(visited, 0, (size_t)n);
        graph g = {adj, deg, R, NULL};
        metric m = {base, d, base + u * d, NULL};
        int64_t ne = 0, nd = 0;
        int32_t size = alg1(&g, &m, nav, l, S, visited, NULL, NULL, 0, &ne, &nd);
        int32_t s = -1;
        for (int32_t t = 0; t < size && s < 0; ++t)
            if (deg[S[t].id] < R) s = S[t].id;
        for (int64_t t = 0; t < n && s < 0; ++t)
            if (reached[t] && deg[t] < R) s = (int32_t)t;
        if (s < 0) {
            rc = ORC_EDEGREE;
            break;
        }
        adj[(int64_t)s * R + deg[s]] = (int32_t)u;
        deg[s] += 1;
        if (added && count < added_cap) {
            added[2 * count] = s;
            added[2 * count + 1] = (int32_t)u;
        }
        count++;
        mark_reachable(adj, deg, R, (int32_t)u, reached, queue);
    }
    if (n_added) *n_added = count;
    free(reached);
    free(queue);
    free(S);
    free(visited);
    return rc;
}

typedef struct {
    const graph *knn;
    const int32_t *knn_ids;
    int32_t K;
    const float *base;
    int64_t n;
    int32_t d, nav, l, C, R;
    int32_t *adj, *deg;
} build_ctx;

static void build_unit(void *p, int64_t v) {
    build_ctx *c = (build_ctx *)p;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * c->C);
    float *dist = (float *)malloc(sizeof(float) * c->C);
    int32_t cnt = collect(c->knn, c->knn_ids + v * c->K, c->K, c->base, c->n, c->d, c->nav,
                          (int32_t)v, c->l, c->C, ids, dist, NULL, NULL);
    c->deg[v] = mrng_select(c->base, c->d, ids, dist, cnt, c->R, c->adj + v * c->R);
    free(ids);
    free(dist);
}

/* Alg. 2's per-node collect and select for every node, given the kNN graph and navigating node. */
int orc_select_all(const int32_t *knn, int32_t K, const float *base, int64_t n, int32_t d,
                   int32_t nav, int32_t l, int32_t R, int32_t C, int32_t nthreads, int32_t *adj,
                   int32_t *deg) {
    if (!knn || !base || !adj || !deg || C < R) return ORC_EINVAL;
    graph g = {knn, NULL, K, NULL};
    build_ctx c = {&g, knn, K, base, n, d, nav, l, C, R, adj, deg};
    run_units(build_unit, &c, n, nthreads);
    return ORC_OK;
}

/*
 * Whole Alg. 2 on the exact kNN graph: kNN -> centroid -> navigating node ->
 * search-collect-select per node -> connectivity.  knn_out ([n][K]) receives
 * the kNN graph when non-NULL.
 */
/* Alg. 2 after its kNN input: centroid, navigating node, search-collect-
 * select for every node, connectivity, on the given kNN graph knn [n][K]. */
int orc_build_on_knn(const float *base, int64_t n, int32_t d, const int32_t *knn, int32_t K, int32_t l,
                     int32_t R, int32_t C, uint64_t seed, int32_t nthreads, int32_t *adj, int32_t *deg,
                     int32_t *nav_out, int32_t *n_added) {
    if (!base || !knn || !adj || !deg || !nav_out || n < 2 || d < 1 || K < 1 || K >= n || l < 1 || R < 1 ||
        C < R)
        return ORC_EINVAL;
    double *c = (double *)malloc(sizeof(double) * d);
    int rc = orc_centroid(base, n, d, c);
    int32_t r = (int32_t)(orc_splitmix64(seed) % (uint64_t)n);
    int32_t nav = 0;
    if (!rc) rc = orc_navigate(knn, n, K, base, d, c, r, l, &nav);
    if (!rc) rc = orc_select_all(knn, K, base, n, d, nav, l, R, C, nthreads, adj, deg);
    if (!rc) rc = orc_connect(adj, deg, n, R, base, d, nav, l, n_added, NULL, 0);
    *nav_out = nav;
    free(c);
    return rc;
}

int orc_build(const float *base, int64_t n, int32_t d, int32_t K, int32_t l, int32_t R, int32_t C,
              uint64_t seed, int32_t nthreads, int32_t *adj, int32_t *deg, int32_t *nav_out,
              int32_t *n_added, int32_t *knn_out) {
    if (!base || !adj || !deg || !nav_out || n < 2 || d < 1 || K < 1 || K >= n || l < 1 ||
        R < 1 || C < R)
        return ORC_EINVAL;
    int32_t *knn = knn_out ? knn_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)n * K);
    int rc = orc_knn_rows(base, n, d, K, NULL, n, nthreads, knn, NULL);
    if (!rc) rc = orc_build_on_knn(base, n, d, knn, K, l, R, C, seed, nthreads, adj, deg, nav_out, n_added);
    if (!knn_out) free(knn);
    return rc;
}

/* NSG-Naive (Section 4.1.2): the MRNG edge selection applied directly to the
 * edges of the kNN graph (each node's K nearest, in key order, are its
 * candidates); no navigating node, no connectivity pass. */
int orc_build_naive(const float *base, int64_t n, int32_t d, int32_t K, int32_t R, int32_t nthreads,
                    int32_t *adj, int32_t *deg) {
    if (!base || !adj || !deg || n < 2 || d < 1 || K < 1 || K >= n || R < 1) return ORC_EINVAL;
    int32_t *knn = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * K);
    float *kd = (float *)malloc(sizeof(float) * (size_t)n * K);
    int rc = orc_knn_rows(base, n, d, K, NULL, n, nthreads, knn, kd);
    for (int64_t v = 0; !rc && v < n; ++v)
        deg[v] = mrng_select(base, d, knn + v * K, kd + v * K, K, R, adj + v * R);
    free(knn);
    free(kd);
    return rc;
}

/* Naive MRNG construction (Section 3.4): every other node is a candidate,
 * no degree cap.  adj is [n][n-1], -1 padded. */
int orc_mrng_naive(const float *base, int64_t n, int32_t d, int32_t *adj, int32_t *deg) {
    if (!base || !adj || !deg || n < 2) return ORC_EINVAL;
    int32_t w = (int32_t)n - 1;
    entry *all = (entry *)malloc(sizeof(entry) * w);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * w);
    float *dist = (float *)malloc(sizeof(float) * w);
    for (int64_t p = 0; p < n; ++p) {
        int32_t c = 0;
        for (int64_t q = 0; q < n; ++q) {
            if (q == p) continue;
            all[c].dist = (double)orc_dist2(base + p * d, base + q * d, d);
            all[c].id = (int32_t)q;
            all[c].checked = 0;
            c++;
        }
        qsort(all, c, sizeof(entry), entry_cmp);
        for (int32_t t = 0; t < c; ++t) {
            ids[t] = all[t].id;
            dist[t] = (float)all[t].dist;
        }
        deg[p] = mrng_select(base, d, ids, dist, c, w, adj + p * w);
    }
    free(all);
    free(ids);
    free(dist);
    return ORC_OK;
}

/* precision (Eq. 1): |R' n R| / K per query, summed hits returned. */
int64_t orc_recall_hits(const int32_t *ids, int32_t ld_ids, const int32_t *gt, int32_t ld_gt,
                        int64_t nq, int32_t k) {
    int64_t hits = 0;
    for (int64_t q = 0; q < nq; ++q)
        for (int32_t a = 0; a < k; ++a) {
            int32_t id = ids[q * ld_ids + a];
            if (id < 0) continue;
            for (int32_t b = 0; b < k; ++b)
                if (gt[q * ld_gt + b] == id) {
                    hits++;
                    break;
                }
        }
    return hits;
}

/* ------------------------------------------------------------------------ */
/* Approximate kNN graph by nn-descent (the approximate kNN graph the build  */
/* starts from, Sec. 3.5 (ii) and the indexing-complexity paragraph of       */
/* Sec. 3.6, built there with Dong, Charikar and Li's nn-descent).  The      */
/* published method's steps, made deterministic (reading R13):               */
/*   init: node v's list is the first K distinct ids != v among              */
/*         splitmix64(seed + v * 0x9e3779b97f4a7c15 + t) mod n, t = 0, 1, ...*/
/*         every entry flagged new;                                          */
/*   each iteration, on the lists as they stand at its start:                */
/*     1. newS(v) = the first S entries of v's list flagged new (key order), */
/*        oldS(v) = the first S flagged old; newS entries become old;        */
/*     2. reverse samples: rnew(u) = the Sr smallest keys (d(u,v), v) over   */
/*        {v : u in newS(v)}, rold(u) likewise over oldS;                    */
/*     3. NEW(v) = newS(v) u rnew(v), OLD(v) = (oldS(v) u rold(v)) \ NEW(v); */
/*     4. local join: for every v, every p in NEW(v) and every q != p in     */
/*        NEW(v) u OLD(v): q is offered to p and p to q, with key d(p, q);   */
/*     5. each list becomes the K smallest keys of itself and its offers     */
/*        (distinct ids); entries that were not in it are flagged new, and   */
/*        their number is the iteration's update count;                      */
/*   stop after `iters` iterations or once an iteration updates at most      */
/*   delta * n * K entries.                                                  */
/* The whole join of an iteration is computed first and the lists replaced  */
/* afterwards, so no step depends on the order of the offers.               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double dist;
    int32_t id;
    int32_t isnew;
} nd_entry;

static int nd_cmp(const void *pa, const void *pb) {
    const nd_entry *a = (const nd_entry *)pa, *b = (const nd_entry *)pb;
    if (a->dist < b->dist) return -1;
    if (a->dist > b->dist) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* offers to one node: a growable array */
typedef struct {
    nd_entry *e;
    int64_t size, cap;
} nd_vec;

static int nd_push(nd_vec *v, double dist, int32_t id, int32_t isnew) {
    if (v->size == v->cap) {
        int64_t c = v->cap ? 2 * v->cap : 16;
        nd_entry *p = (nd_entry *)realloc(v->e, sizeof(nd_entry) * (size_t)c);
        if (!p) return ORC_ENOMEM;
        v->e = p;
        v->cap = c;
    }
    v->e[v->size].dist = dist;
    v->e[v->size].id = id;
    v->e[v->size].isnew = isnew;
    v->size++;
    return ORC_OK;
}

static int nd_has(const int32_t *ids, int32_t m, int32_t id) {
    for (int32_t i = 0; i < m; ++i)
        if (ids[i] == id) return 1;
    return 0;
}

/* ids [n][K], dist [n][K] out (sorted by key); *iters_run and *last_updates
 * (nullable) report the iterations run and the last iteration's updates. */
int orc_nndescent(const float *base, int64_t n, int32_t d, int32_t K, int32_t S, int32_t Sr, int32_t iters,
                  float delta, uint64_t seed, int32_t *ids, float *dist, int32_t *iters_run,
                  int64_t *last_updates) {
    if (!base || !ids || n < 2 || d < 1 || K < 1 || K >= n || S < 0 || Sr < 0 || iters < 0) return ORC_EINVAL;
    nd_entry *list = (nd_entry *)malloc(sizeof(nd_entry) * (size_t)n * K);
    int32_t *newS = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (S > 0 ? S : 1));
    int32_t *oldS = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (S > 0 ? S : 1));
    int32_t *nnew = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *nold = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    nd_vec *rnew = (nd_vec *)calloc((size_t)n, sizeof(nd_vec));
    nd_vec *rold = (nd_vec *)calloc((size_t)n, sizeof(nd_vec));
    nd_vec *offers = (nd_vec *)calloc((size_t)n, sizeof(nd_vec));
    int32_t cap = 2 * (S + Sr) + 2;
    int32_t *NEWv = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *OLDv = (int32_t *)malloc(sizeof(int32_t) * cap);
    nd_entry *merged = (nd_entry *)malloc(sizeof(nd_entry) * (size_t)K);
    int rc = ORC_OK;
    if (!list || !newS || !oldS || !nnew || !nold || !rnew || !rold || !offers || !NEWv || !OLDv || !merged)
        rc = ORC_ENOMEM;
    /* init: K distinct random ids per node */
    for (int64_t v = 0; !rc && v < n; ++v) {
        nd_entry *L = list + v * K;
        int32_t m = 0;
        int32_t *got = (int32_t *)malloc(sizeof(int32_t) * K);
        for (uint64_t t = 0; m < K; ++t) {
            int32_t x = (int32_t)(orc_splitmix64(seed + (uint64_t)v * 0x9e3779b97f4a7c15ULL + t) % (uint64_t)n);
            if (x == v || nd_has(got, m, x)) continue;
            got[m] = x;
            L[m].dist = (double)orc_dist2(base + v * d, base + (int64_t)x * d, d);
            L[m].id = x;
            L[m].isnew = 1;
            m++;
        }
        free(got);
        qsort(L, K, sizeof(nd_entry), nd_cmp);
    }
    int32_t it = 0;
    int64_t updates = 0;
    for (; !rc && it < iters; ++it) {
        /* 1. samples */
        for (int64_t v = 0; v < n; ++v) {
            nd_entry *L = list + v * K;
            nnew[v] = nold[v] = 0;
            for (int32_t i = 0; i < K; ++i) {
                if (L[i].isnew && nnew[v] < S) newS[v * S + nnew[v]++] = L[i].id;
                else if (!L[i].isnew && nold[v] < S) oldS[v * S + nold[v]++] = L[i].id;
            }
            for (int32_t i = 0; i < K; ++i)
                if (L[i].isnew && nd_has(newS + v * S, nnew[v], L[i].id)) L[i].isnew = 0;
        }
        /* 2. reverse samples (all, then the Sr smallest keys per node) */
        for (int64_t v = 0; v < n; ++v) {
            rnew[v].size = rold[v].size = 0;
            offers[v].size = 0;
        }
        for (int64_t v = 0; !rc && v < n; ++v) {
            const nd_entry *L = list + v * K;
            for (int32_t i = 0; !rc && i < K; ++i) {
                const int32_t u = L[i].id;
                if (nd_has(newS + v * S, nnew[v], u)) rc = nd_push(&rnew[u], L[i].dist, (int32_t)v, 1);
                else if (nd_has(oldS + v * S, nold[v], u)) rc = nd_push(&rold[u], L[i].dist, (int32_t)v, 0);
            }
        }
        for (int64_t u = 0; !rc && u < n; ++u) {
            qsort(rnew[u].e, rnew[u].size, sizeof(nd_entry), nd_cmp);
            qsort(rold[u].e, rold[u].size, sizeof(nd_entry), nd_cmp);
            if (rnew[u].size > Sr) rnew[u].size = Sr;
            if (rold[u].size > Sr) rold[u].size = Sr;
        }
        /* 3 + 4. join sets and the local join, offers collected per node */
        for (int64_t v = 0; !rc && v < n; ++v) {
            int32_t a = 0, b = 0;
            for (int32_t i = 0; i < nnew[v]; ++i)
                if (!nd_has(NEWv, a, newS[v * S + i])) NEWv[a++] = newS[v * S + i];
            for (int64_t i = 0; i < rnew[v].size; ++i)
                if (!nd_has(NEWv, a, rnew[v].e[i].id)) NEWv[a++] = rnew[v].e[i].id;
            for (int32_t i = 0; i < nold[v]; ++i)
                if (!nd_has(NEWv, a, oldS[v * S + i]) && !nd_has(OLDv, b, oldS[v * S + i])) OLDv[b++] = oldS[v * S + i];
            for (int64_t i = 0; i < rold[v].size; ++i)
                if (!nd_has(NEWv, a, rold[v].e[i].id) && !nd_has(OLDv, b, rold[v].e[i].id)) OLDv[b++] = rold[v].e[i].id;
            for (int32_t i = 0; !rc && i < a; ++i) {
                const int32_t p = NEWv[i];
                for (int32_t j = 0; !rc && j < a + b; ++j) {
                    const int32_t q = j < a ? NEWv[j] : OLDv[j - a];
                    if (q == p) continue;
                    const double dd = (double)orc_dist2(base + (int64_t)p * d, base + (int64_t)q * d, d);
                    rc = nd_push(&offers[p], dd, q, 1);
                    if (!rc) rc = nd_push(&offers[q], dd, p, 1);
                }
            }
        }
        /* 5. each list: the K smallest of itself and its offers, distinct ids */
        updates = 0;
        for (int64_t p = 0; !rc && p < n; ++p) {
            nd_entry *L = list + p * K;
            nd_vec *o = &offers[p];
            qsort(o->e, o->size, sizeof(nd_entry), nd_cmp);
            int32_t m = 0, i = 0;
            int64_t j = 0;
            while (m < K && (i < K || j < o->size)) {
                nd_entry e;
                if (j >= o->size || (i < K && nd_cmp(&L[i], &o->e[j]) <= 0)) e = L[i++];
                else e = o->e[j++];
                /* an id offered again, or offered while in the list (same key: the
                 * list's own entry, with its flag, comes first) is kept once */
                int dup = 0;
                for (int32_t t = 0; t < m; ++t)
                    if (merged[t].id == e.id) dup = 1;
                if (dup) continue;
                merged[m++] = e;
            }
            for (int32_t t = 0; t < K; ++t) {
                int was = 0;
                for (int32_t r = 0; r < K; ++r)
                    if (L[r].id == merged[t].id) was = 1;
                if (!was) updates++;
            }
            memcpy(L, merged, sizeof(nd_entry) * (size_t)K);
        }
        if (!rc && updates <= (int64_t)((double)delta * (double)n * (double)K)) {
            ++it;
            break;
        }
    }
    for (int64_t v = 0; !rc && v < n; ++v)
        for (int32_t i = 0; i < K; ++i) {
            ids[v * K + i] = list[v * K + i].id;
            if (dist) dist[v * K + i] = (float)list[v * K + i].dist;
        }
    if (iters_run) *iters_run = it;
    if (last_updates) *last_updates = updates;
    for (int64_t v = 0; rnew && v < n; ++v) {
        free(rnew[v].e);
        free(rold[v].e);
        free(offers[v].e);
    }
    free(list);
    free(newS);
    free(oldS);
    free(nnew);
    free(nold);
    free(rnew);
    free(rold);
    free(offers);
    free(NEWv);
    free(OLDv);
    free(merged);
    return rc;
}
