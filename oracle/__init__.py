"""CPU oracle for the NSG hot path (ctypes wrapper around ``nsg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle shares no code
with the CUDA path and never calls it; the CUDA path never imports this
package.  Each function below names the part of the paper it computes; the C
file header lists the readings taken where the paper is silent or garbled.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# Plain C, no FMA contraction, no fast-math: the float sums follow the source order.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-pthread"]

_lib = None


def compile_lib(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(compile_lib())
        _decl(_lib)
    return _lib


P = C.c_void_p
i32, i64, u64, f32 = C.c_int32, C.c_int64, C.c_uint64, C.c_float


def _decl(L):
    L.orc_dist2.argtypes = [P, P, i32]
    L.orc_dist2.restype = f32
    L.orc_knn_rows.argtypes = [P, i64, i32, i32, P, i64, i32, P, P]
    L.orc_knn_query.argtypes = [P, i64, i32, P, i64, i32, i32, P, P]
    L.orc_lazy_knn_new.argtypes = [P, i64, i32, i32, i32]
    L.orc_lazy_knn_new.restype = P
    L.orc_lazy_knn_free.argtypes = [P]
    L.orc_lazy_knn_row.argtypes = [P, i32]
    L.orc_lazy_knn_row.restype = P
    L.orc_lazy_knn_rows_computed.argtypes = [P]
    L.orc_lazy_knn_rows_computed.restype = i64
    L.orc_search.argtypes = [P, P, i64, i32, P, i32, i32, P, i64, i32, i32, i32, P, P, P, P]
    L.orc_search_trace.argtypes = [P, P, i64, i32, P, i32, i32, P, i32, P, i32, P]
    L.orc_splitmix64.argtypes = [u64]
    L.orc_splitmix64.restype = u64
    L.orc_centroid.argtypes = [P, i64, i32, P]
    L.orc_navigate.argtypes = [P, i64, i32, P, i32, P, i32, i32, P]
    L.orc_navigate_lazy.argtypes = [P, P, i32, i32, P]
    L.orc_prune.argtypes = [P, i32, P, P, i32, i32, P, P]
    L.orc_collect.argtypes = [P, i32, P, i64, i32, i32, i32, i32, i32, P, P, P, P, P]
    L.orc_collect_lazy.argtypes = [P, i32, i32, i32, i32, P, P, P]
    L.orc_connect.argtypes = [P, P, i64, i32, P, i32, i32, i32, P, P, i32]
    L.orc_select_all.argtypes = [P, i32, P, i64, i32, i32, i32, i32, i32, i32, P, P]
    L.orc_build.argtypes = [P, i64, i32, i32, i32, i32, i32, u64, i32, P, P, P, P, P]
    L.orc_mrng_naive.argtypes = [P, i64, i32, P, P]
    L.orc_build_naive.argtypes = [P, i64, i32, i32, i32, i32, P, P]
    L.orc_search_random.argtypes = [P, P, i64, i32, P, i32, P, i64, i32, i32, i32, u64, i32, P, P, P, P]
    L.orc_build_on_knn.argtypes = [P, i64, i32, P, i32, i32, i32, i32, u64, i32, P, P, P, P]
    L.orc_nndescent.argtypes = [P, i64, i32, i32, i32, i32, i32, f32, u64, P, P, P, P]
    L.orc_recall_hits.argtypes = [P, i32, P, i32, i64, i32]
    L.orc_recall_hits.restype = i64


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


def dist2(a, b) -> float:
    """Squared l2 distance, float32, summed in index order (Section 2)."""
    a, b = _f32(a), _f32(b)
    return float(lib().orc_dist2(_p(a), _p(b), a.shape[-1]))


def knn_rows(base, K, rows=None, nthreads=None):
    """kNN graph rows by serial scan, self excluded by id (Alg. 2 input)."""
    base = _f32(base)
    n, d = base.shape
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if r is None else len(r)
    ids = np.empty((nr, K), np.int32)
    dist = np.empty((nr, K), np.float32)
    _check(lib().orc_knn_rows(_p(base), n, d, K, _p(r), nr, nthreads or nthreads_default(),
                              _p(ids), _p(dist)), "knn_rows")
    return ids, dist


def knn_query(base, queries, k, nthreads=None):
    """Exact k nearest base rows per query (serial scan, Section 4.1.2)."""
    base, queries = _f32(base), _f32(queries)
    n, d = base.shape
    nq = len(queries)
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    _check(lib().orc_knn_query(_p(base), n, d, _p(queries), nq, k, nthreads or nthreads_default(),
                               _p(ids), _p(dist)), "knn_query")
    return ids, dist


def search(adj, base, start, queries, k, L, deg=None, nthreads=1):
    """Alg. 1 from ``start`` on a fixed-width graph; returns ids, dists,
    n_expand (nodes checked), n_dist (distances computed)."""
    adj, base, queries = _i32(adj), _f32(base), _f32(queries)
    n, width = adj.shape
    d = base.shape[1]
    dg = None if deg is None else _i32(deg)
    nq = len(queries)
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    ne = np.empty(nq, np.int64)
    nd = np.empty(nq, np.int64)
    _check(lib().orc_search(_p(adj), _p(dg), n, width, _p(base), d, int(start), _p(queries), nq,
                            k, L, nthreads, _p(ids), _p(dist), _p(ne), _p(nd)), "search")
    return ids, dist, ne, nd


def search_trace(adj, base, start, q, L, max_steps=1000, deg=None):
    """Pool ids after each expansion of Alg. 1 (one query)."""
    adj, base, q = _i32(adj), _f32(base), _f32(q)
    n, width = adj.shape
    dg = None if deg is None else _i32(deg)
    trace = np.full((max_steps, L), -1, np.int32)
    steps = C.c_int64(0)
    _check(lib().orc_search_trace(_p(adj), _p(dg), n, width, _p(base), base.shape[1], int(start),
                                  _p(q), L, _p(trace), max_steps, C.byref(steps)), "search_trace")
    return trace[:min(steps.value, max_steps)]


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x))


def start_node(seed: int, n: int) -> int:
    """Random start node of Alg. 2: splitmix64(seed) mod n (reading R5)."""
    return splitmix64(seed) % n


def centroid(base):
    """Centroid step of Alg. 2: mean row in double."""
    base = _f32(base)
    n, d = base.shape
    c = np.empty(d, np.float64)
    _check(lib().orc_centroid(_p(base), n, d, _p(c)), "centroid")
    return c


def navigate(knn, base, c, r, L):
    """Navigating-node step of Alg. 2: from start r toward centroid c."""
    knn, base = _i32(knn), _f32(base)
    c = np.ascontiguousarray(c, np.float64)
    nav = C.c_int32(0)
    _check(lib().orc_navigate(_p(knn), knn.shape[0], knn.shape[1], _p(base), base.shape[1], _p(c),
                              int(r), L, C.byref(nav)), "navigate")
    return nav.value


def collect(knn, base, nav, v, L, Cap):
    """Search-and-collect step of Alg. 2 for node v: (ids, dists, count, n_expand, n_dist)."""
    knn, base = _i32(knn), _f32(base)
    ids = np.empty(Cap, np.int32)
    dist = np.empty(Cap, np.float32)
    cnt = C.c_int32(0)
    ne, nd = C.c_int64(0), C.c_int64(0)
    _check(lib().orc_collect(_p(knn), knn.shape[1], _p(base), base.shape[0], base.shape[1], int(nav),
                             int(v), L, Cap, _p(ids), _p(dist), C.byref(cnt), C.byref(ne),
                             C.byref(nd)), "collect")
    return ids, dist, cnt.value, ne.value, nd.value


def prune(base, cand_ids, cand_dist, R):
    """MRNG edge selection of Alg. 2; returns (row [R] -1 padded, deg)."""
    base = _f32(base)
    ci, cd = _i32(cand_ids), _f32(cand_dist)
    ncand = int(np.sum(ci >= 0)) if len(ci) else 0
    out = np.empty(R, np.int32)
    deg = C.c_int32(0)
    _check(lib().orc_prune(_p(base), base.shape[1], _p(ci), _p(cd), ncand, R, _p(out),
                           C.byref(deg)), "prune")
    return out, deg.value


def select_all(knn, base, nav, L, R, Cap, nthreads=None):
    """Alg. 2's per-node collect and select for every node (before the connectivity pass)."""
    knn, base = _i32(knn), _f32(base)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    _check(lib().orc_select_all(_p(knn), knn.shape[1], _p(base), n, d, int(nav), L, R, Cap,
                                nthreads or nthreads_default(), _p(adj), _p(deg)), "select_all")
    return adj, deg


def connect(adj, deg, base, nav, L, added_cap=1 << 16):
    """Connectivity step of Alg. 2 on copies of adj/deg; returns (adj, deg, added [m][2])."""
    adj = np.array(adj, dtype=np.int32, copy=True, order="C")
    deg = np.array(deg, dtype=np.int32, copy=True, order="C")
    base = _f32(base)
    n, R = adj.shape
    added = np.empty((added_cap, 2), np.int32)
    cnt = C.c_int32(0)
    rc = lib().orc_connect(_p(adj), _p(deg), n, R, _p(base), base.shape[1], int(nav), L,
                           C.byref(cnt), _p(added), added_cap)
    _check(rc, "connect")
    return adj, deg, added[:min(cnt.value, added_cap)].copy()


def build(base, K, L, R, Cap, seed=0, nthreads=None):
    """Whole Alg. 2 on the exact kNN graph.  Returns dict(adj, deg, nav, n_added, knn)."""
    base = _f32(base)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    knn = np.empty((n, K), np.int32)
    nav = C.c_int32(0)
    added = C.c_int32(0)
    _check(lib().orc_build(_p(base), n, d, K, L, R, Cap, seed, nthreads or nthreads_default(),
                           _p(adj), _p(deg), C.byref(nav), C.byref(added), _p(knn)), "build")
    return dict(adj=adj, deg=deg, nav=nav.value, n_added=added.value, knn=knn)


def build_on_knn(base, knn, L, R, Cap, seed=0, nthreads=None):
    """Alg. 2 after its kNN input, on a given kNN graph knn [n][K] (e.g. an
    approximate one).  Returns dict(adj, deg, nav, n_added)."""
    base = _f32(base)
    knn = _i32(knn)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    nav = C.c_int32(0)
    added = C.c_int32(0)
    _check(lib().orc_build_on_knn(_p(base), n, d, _p(knn), knn.shape[1], L, R, Cap, seed,
                                  nthreads or nthreads_default(), _p(adj), _p(deg), C.byref(nav), C.byref(added)),
           "build_on_knn")
    return dict(adj=adj, deg=deg, nav=nav.value, n_added=added.value)


def build_naive(base, K, R, nthreads=None):
    """NSG-Naive (Section 4.1.2): MRNG edge selection over each node's K
    nearest neighbours; no navigating node, no connectivity pass.  Returns
    (adj [n][R] -1 padded, deg [n])."""
    base = _f32(base)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    _check(lib().orc_build_naive(_p(base), n, d, K, R, nthreads or nthreads_default(), _p(adj), _p(deg)),
           "build_naive")
    return adj, deg


def search_random(adj, base, queries, k, L, count, seed, deg=None, nthreads=1):
    """Alg. 1 whose pool starts as the set of `count` seeded random nodes
    (query q draws splitmix64(seed + q * 0x9e3779b97f4a7c15 + j) mod n, j < count).
    Returns ids, dists, n_expand, n_dist like `search`."""
    adj, base, queries = _i32(adj), _f32(base), _f32(queries)
    n, width = adj.shape
    d = base.shape[1]
    dg = None if deg is None else _i32(deg)
    nq = len(queries)
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float32)
    ne = np.empty(nq, np.int64)
    nd = np.empty(nq, np.int64)
    _check(lib().orc_search_random(_p(adj), _p(dg), n, width, _p(base), d, _p(queries), nq, k, L, count,
                                   seed, nthreads, _p(ids), _p(dist), _p(ne), _p(nd)), "search_random")
    return ids, dist, ne, nd


def partition_search(base, queries, part, K, L_build, R, Cap, k, L, seed=0, nthreads=None):
    """Partition-and-merge search (Sections 4.2, 4.3): the base is split into
    subsets (``part[i]`` = row i's subset), one NSG is built per subset (Alg. 2
    on that subset's rows, ids local to it, kNN degree min(K, size - 1)),
    every query runs Alg. 1 on every subset's NSG with pool L (returning
    min(k, size) results), the local ids are mapped back to row ids, and the
    union is cut to the k smallest keys (distance, row id).  Every subset
    needs at least 2 rows.  Returns (ids [nq][k], d2 [nq][k]), padded with
    -1 / +inf when the subsets hold fewer than k rows in all."""
    base, queries = _f32(base), _f32(queries)
    part = np.asarray(part)
    if part.shape != (len(base),):
        raise ValueError("part needs one subset id per base row")
    if np.unique(part, return_counts=True)[1].min() < 2:
        raise ValueError("every subset needs at least 2 rows")
    nq = len(queries)
    gids, dists = [], []
    for p in np.unique(part):
        rows = np.flatnonzero(part == p).astype(np.int32)
        sub = base[rows]
        g = build(sub, min(K, len(rows) - 1), L_build, R, Cap, seed=seed, nthreads=nthreads)
        kp = min(k, len(rows))
        ids, d2, _, _ = search(g["adj"], sub, g["nav"], queries, kp, max(L, kp), deg=g["deg"],
                               nthreads=nthreads or nthreads_default())
        gids.append(np.where(ids >= 0, rows[np.maximum(ids, 0)], -1).astype(np.int32))
        dists.append(np.where(ids >= 0, d2, np.float32(np.inf)).astype(np.float32))
    gid, dist = np.concatenate(gids, axis=1), np.concatenate(dists, axis=1)
    out_ids = np.full((nq, k), -1, np.int32)
    out_d2 = np.full((nq, k), np.inf, np.float32)
    for q in range(nq):
        # key order: distance, then row id; padding (+inf) sorts last
        order = np.lexsort((np.where(gid[q] >= 0, gid[q], np.iinfo(np.int32).max), dist[q]))[:k]
        m = len(order)
        out_ids[q, :m], out_d2[q, :m] = gid[q, order], dist[q, order]
    return out_ids, out_d2


def nndescent(base, K, S=16, Sr=16, iters=10, delta=0.001, seed=0):
    """Approximate kNN graph by nn-descent (the approximate kNN graph the build
    starts from, Sec. 3.5 (ii); Dong, Charikar and Li's method made
    deterministic: seeded random init, per iteration S sampled new / old
    entries and Sr reverse samples per node, local join, each list cut to its
    K smallest keys).  Returns (ids [n][K], d2 [n][K], iterations run,
    updates of the last iteration)."""
    base = _f32(base)
    n, d = base.shape
    ids = np.empty((n, K), np.int32)
    dist = np.empty((n, K), np.float32)
    it = C.c_int32(0)
    upd = C.c_int64(0)
    _check(lib().orc_nndescent(_p(base), n, d, K, S, Sr, iters, delta, seed, _p(ids), _p(dist), C.byref(it),
                               C.byref(upd)), "nndescent")
    return ids, dist, it.value, upd.value


def mrng_naive(base):
    """Naive MRNG construction (Section 3.4); adj [n][n-1] -1 padded, deg [n]."""
    base = _f32(base)
    n, d = base.shape
    adj = np.empty((n, n - 1), np.int32)
    deg = np.empty(n, np.int32)
    _check(lib().orc_mrng_naive(_p(base), n, d, _p(adj), _p(deg)), "mrng_naive")
    return adj, deg


def recall(ids, gt, k):
    """Mean precision (Eq. 1) of the first k ids against the first k ground-truth ids."""
    ids, gt = _i32(ids), _i32(gt)
    nq = len(ids)
    hits = lib().orc_recall_hits(_p(ids), ids.shape[1], _p(gt), gt.shape[1], nq, k)
    return hits / float(nq * k)


class LazyKnn:
    """kNN graph whose rows are computed by serial scan on first use, so the
    oracle can follow a search over a large base one row at a time."""

    def __init__(self, base, K, nthreads=None):
        self.base = _f32(base)
        n, d = self.base.shape
        self.h = lib().orc_lazy_knn_new(_p(self.base), n, d, K, nthreads or nthreads_default())
        self.K = K

    def row(self, u):
        p = lib().orc_lazy_knn_row(self.h, int(u))
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_int32)), shape=(self.K,)).copy()

    def rows_computed(self):
        return int(lib().orc_lazy_knn_rows_computed(self.h))

    def navigate(self, c, r, L):
        c = np.ascontiguousarray(c, np.float64)
        nav = C.c_int32(0)
        _check(lib().orc_navigate_lazy(self.h, _p(c), int(r), L, C.byref(nav)), "navigate_lazy")
        return nav.value

    def collect(self, nav, v, L, Cap):
        ids = np.empty(Cap, np.int32)
        dist = np.empty(Cap, np.float32)
        cnt = C.c_int32(0)
        _check(lib().orc_collect_lazy(self.h, int(nav), int(v), L, Cap, _p(ids), _p(dist),
                                      C.byref(cnt)), "collect_lazy")
        return ids, dist, cnt.value

    def __del__(self):
        try:
            lib().orc_lazy_knn_free(self.h)
        except Exception:
            pass
