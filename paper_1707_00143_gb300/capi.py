"""Thin ctypes binding of ``libnsg.so`` (declared in ``include/nsg.h``).

Argument marshalling only: tensors become raw device pointers, the current
torch stream becomes the ``stream`` argument, status codes become
exceptions.  Every step of the method runs in the library's CUDA kernels.
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnsg.so")

NSG_OK, NSG_EINVAL, NSG_ENOMEM, NSG_ECUDA, NSG_ESTEPCAP, NSG_EDEGREE, NSG_EIO, NSG_EFORMAT = (
    0, -1, -2, -3, -4, -5, -6, -7)
PREC_F32, PREC_BF16, PREC_FP8, PREC_U8 = 0, 1, 2, 3


class NsgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib().nsg_status_str(status).decode()
        if status == NSG_ECUDA:
            msg += " (" + lib().nsg_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")


class SearchParams(C.Structure):
    """nsg_search_params (include/nsg.h has each field's full meaning).  Zero
    leaves a choice to the library: max_steps (16 L + 4096), hash_slots (sized
    to the batch), warps_per_cta, warps_per_query and stage_rows (measured
    rules), pool (shared memory up to L = 1024); rerank -1 re-ranks only lossy
    copies.  stop_model: a device tensor of NSG_STOP_PARAMS FP16 values or None.
    None of those automatic choices (hash_slots, warps_per_cta, warps_per_query,
    stage_rows, pool) changes a query's result."""
    _fields_ = [("max_steps", C.c_int32), ("hash_slots", C.c_int32), ("precision", C.c_int32),
                ("warps_per_cta", C.c_int32), ("rerank", C.c_int32), ("stop_model", C.c_void_p),
                ("stop_threshold", C.c_float), ("stop_k", C.c_int32), ("stop_min_steps", C.c_int32),
                ("init_random", C.c_int32), ("init_seed", C.c_uint64), ("warps_per_query", C.c_int32),
                ("pool", C.c_int32), ("stage_rows", C.c_int32)]

    def __init__(self, max_steps=0, hash_slots=0, precision=0, warps_per_cta=0, rerank=-1, stop_model=None,
                 stop_threshold=0.5, stop_k=0, stop_min_steps=0, init_random=0, init_seed=0, warps_per_query=0,
                 pool=0, stage_rows=0):
        ptr = stop_model.data_ptr() if isinstance(stop_model, torch.Tensor) else stop_model
        super().__init__(max_steps, hash_slots, precision, warps_per_cta, rerank, ptr, stop_threshold, stop_k,
                         stop_min_steps, init_random, init_seed, warps_per_query, pool, stage_rows)


STOP_FEATURES, STOP_PARAMS = 8, 641
POOL_AUTO, POOL_SHARED, POOL_GLOBAL = 0, 1, 2
MAX_L = 8192
STAGE_MAX = 32  # staged row gathers: most rows in flight per warp (SearchParams.stage_rows)


class NnDescentParams(C.Structure):
    """nn-descent settings: samples per list, reverse samples per node,
    iteration cap, stopping fraction, seed of the initial lists."""
    _fields_ = [("sample", C.c_int32), ("reverse", C.c_int32), ("iters", C.c_int32), ("delta", C.c_float),
                ("seed", C.c_uint64)]

    def __init__(self, sample=16, reverse=16, iters=10, delta=0.001, seed=0):
        super().__init__(sample, reverse, iters, delta, seed)


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("R", C.c_int32), ("nav", C.c_int32),
                ("max_degree", C.c_int32), ("avg_degree", C.c_double), ("n_fixup_edges", C.c_int64),
                ("device_bytes", C.c_int64), ("has_bf16", C.c_int32), ("has_fp8", C.c_int32),
                ("fp8_scale", C.c_float), ("ms_knn", C.c_float), ("ms_centroid_nav", C.c_float),
                ("ms_collect", C.c_float), ("ms_prune", C.c_float), ("ms_connect", C.c_float),
                ("ms_total", C.c_float), ("n_fixup_searches", C.c_int64), ("has_u8", C.c_int32),
                ("u8_lo", C.c_float), ("u8_scale", C.c_float), ("prune_examined", C.c_int64),
                ("parts", C.c_int32), ("knn_iters", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
P, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64

# (name, argtypes, restype) of every exported symbol -- the same list as include/nsg.h
SIGNATURES = [
    ("nsg_status_str", [i32], C.c_char_p),
    ("nsg_last_cuda_error", [], C.c_char_p),
    ("nsg_knn_init", [P, i64, i32, i32, P, P, P], i32),
    ("nsg_knn_query", [P, i64, i32, P, i64, i32, P, P, P], i32),
    ("nsg_centroid", [P, i64, i32, P, P], i32),
    ("nsg_navigate", [P, i64, i32, P, i32, P, i32, i32, P, P], i32),
    ("nsg_navigate_noalloc", [P, i64, i32, P, i32, P, i32, i32, P, P], i32),
    ("nsg_collect", [P, i64, i32, P, i32, i32, i32, i32, i64, i64, P, P, P, P, P], i32),
    ("nsg_prune", [P, i64, i32, P, P, P, i32, i32, i64, i64, P, P, P], i32),
    ("nsg_connect", [P, i64, i32, P, P, i32, i32, i32, P, P], i32),
    ("nsg_build", [P, i64, i32, i32, i32, i32, i32, u64, P, P], i32),
    ("nsg_build_naive", [P, i64, i32, i32, i32, u64, P, P], i32),
    ("nsg_index_from_graph", [P, i64, i32, P, P, i32, i32, P, P], i32),
    ("nsg_search", [P, P, i64, i32, i32, P, P, P], i32),
    ("nsg_search_ex", [P, P, i64, i32, i32, P, P, P, P, P, P, P], i32),
    ("nsg_search_host", [P, P, i64, i32, i32, P, P, P, P], i32),
    ("nsg_build_partitioned", [P, i64, i32, P, i32, i32, i32, i32, i32, u64, P, P], i32),
    ("nsg_knn_nndescent", [P, i64, i32, i32, P, P, P, P, P, P], i32),
    ("nsg_build_ex", [P, i64, i32, i32, i32, i32, i32, u64, P, P, P], i32),
    ("nsg_search_partitioned", [P, P, i64, i32, i32, P, P, P, P], i32),
    ("nsg_recall", [P, i32, P, i32, i64, i32, P, P], i32),
    ("nsg_search_trace", [P, P, i64, i32, i32, P, P, P, P, P, i32, P], i32),
    ("nsg_search_batched", [P, P, i64, P, P, i32, i32, P, P, P, P, P], i32),
    ("nsg_plan_create", [P, P, i64, P, P, i32, i32, P, P, P, P, i32, P, P], i32),
    ("nsg_plan_run", [P, P], i32),
    ("nsg_plan_info", [P, P], i32),
    ("nsg_plan_free", [P], None),
    ("nsg_stop_train", [P, P, P, i64, i32, i32, C.c_float, u64, P, P, P, P], i32),
    ("nsg_index_info", [P, P], i32),
    ("nsg_index_prepare", [P, i32, P], i32),
    ("nsg_index_graph", [P, P, P, P], i32),
    ("nsg_save", [P, C.c_char_p], i32),
    ("nsg_load", [C.c_char_p, P, P], i32),
    ("nsg_free", [P], None),
]


def lib():
    """Load libnsg.so (built by ``paper_1707_00143_gb300.build``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1707_00143_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, args, res in SIGNATURES:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc, where):
    if rc != NSG_OK:
        raise NsgError(rc, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor")
    return t


def _host(t, dtype):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous host {dtype} tensor")
    return t


def nsg_knn_init(base, K, with_d2=True):
    base = _dev(base, torch.float32)
    n, d = base.shape
    ids = torch.empty((n, K), dtype=torch.int32, device=base.device)
    d2 = torch.empty((n, K), dtype=torch.float32, device=base.device) if with_d2 else None
    _check(lib().nsg_knn_init(_ptr(base), n, d, K, _ptr(ids), _ptr(d2), _stream()), "nsg_knn_init")
    return ids, d2


def nsg_knn_query(base, queries, k):
    base, queries = _dev(base, torch.float32), _dev(queries, torch.float32)
    n, d = base.shape
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=base.device)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=base.device)
    _check(lib().nsg_knn_query(_ptr(base), n, d, _ptr(queries), nq, k, _ptr(ids), _ptr(d2), _stream()),
           "nsg_knn_query")
    return ids, d2


def nsg_centroid(base):
    base = _dev(base, torch.float32)
    n, d = base.shape
    c = torch.empty(d, dtype=torch.float64, device=base.device)
    _check(lib().nsg_centroid(_ptr(base), n, d, _ptr(c), _stream()), "nsg_centroid")
    return c


def nsg_navigate(base, knn, centroid, start, L):
    base, knn = _dev(base, torch.float32), _dev(knn, torch.int32)
    centroid = _dev(centroid, torch.float64)
    n, d = base.shape
    nav = C.c_int32(0)
    _check(lib().nsg_navigate(_ptr(base), n, d, _ptr(knn), knn.shape[1], _ptr(centroid), int(start), L,
                              C.byref(nav), _stream()), "nsg_navigate")
    return nav.value


def nsg_navigate_noalloc(base, knn, centroid, start, L):
    """nsg_navigate for callers that may not allocate device memory: the
    visited bitmap is a fixed array inside the library (n <= 16,777,216);
    calls sharing a device must not overlap on the GPU."""
    base, knn = _dev(base, torch.float32), _dev(knn, torch.int32)
    centroid = _dev(centroid, torch.float64)
    n, d = base.shape
    nav = C.c_int32(0)
    _check(lib().nsg_navigate_noalloc(_ptr(base), n, d, _ptr(knn), knn.shape[1], _ptr(centroid), int(start),
                                      L, C.byref(nav), _stream()), "nsg_navigate_noalloc")
    return nav.value


def nsg_collect(base, knn, nav, L, Cap, v0=0, nv=None):
    base, knn = _dev(base, torch.float32), _dev(knn, torch.int32)
    n, d = base.shape
    nv = n - v0 if nv is None else nv
    dev = base.device
    ids = torch.empty((nv, Cap), dtype=torch.int32, device=dev)
    d2 = torch.empty((nv, Cap), dtype=torch.float32, device=dev)
    cnt = torch.empty(nv, dtype=torch.int32, device=dev)
    st = torch.empty(nv, dtype=torch.int32, device=dev)
    _check(lib().nsg_collect(_ptr(base), n, d, _ptr(knn), knn.shape[1], int(nav), L, Cap, v0, nv,
                             _ptr(ids), _ptr(d2), _ptr(cnt), _ptr(st), _stream()), "nsg_collect")
    return ids, d2, cnt, st


def nsg_prune(base, cand_ids, cand_d2, cand_count, R, v0=0, adj=None, deg=None):
    base = _dev(base, torch.float32)
    n, d = base.shape
    nv, Cap = cand_ids.shape
    dev = base.device
    adj = torch.full((n, R), -1, dtype=torch.int32, device=dev) if adj is None else adj
    deg = torch.zeros(n, dtype=torch.int32, device=dev) if deg is None else deg
    _check(lib().nsg_prune(_ptr(base), n, d, _ptr(_dev(cand_ids, torch.int32)),
                           _ptr(_dev(cand_d2, torch.float32)), _ptr(_dev(cand_count, torch.int32)),
                           Cap, R, v0, nv, _ptr(adj), _ptr(deg), _stream()), "nsg_prune")
    return adj, deg


def nsg_connect(base, adj, deg, nav, L):
    base = _dev(base, torch.float32)
    adj, deg = _dev(adj, torch.int32), _dev(deg, torch.int32)
    n, d = base.shape
    added = C.c_int32(0)
    _check(lib().nsg_connect(_ptr(base), n, d, _ptr(adj), _ptr(deg), adj.shape[1], int(nav), L,
                             C.byref(added), _stream()), "nsg_connect")
    return added.value


def nsg_recall(ids, gt, k):
    ids, gt = _dev(ids, torch.int32), _dev(gt, torch.int32)
    hits = torch.empty(ids.shape[0], dtype=torch.int32, device=ids.device)
    _check(lib().nsg_recall(_ptr(ids), ids.shape[1], _ptr(gt), gt.shape[1], ids.shape[0], k, _ptr(hits),
                            _stream()), "nsg_recall")
    return hits


class Index:
    """Owner of an ``nsg_index*`` (freed with the object or by ``free()``)."""

    def __init__(self, handle):
        self.h = handle

    def free(self):
        if self.h:
            lib().nsg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self):
        inf = IndexInfo()
        _check(lib().nsg_index_info(self.h, C.byref(inf)), "nsg_index_info")
        return inf.as_dict()

    def prepare(self, precision):
        """Build the BF16 (1) or FP8-e4m3 (2) copy used by the precision forms."""
        _check(lib().nsg_index_prepare(self.h, precision, _stream()), "nsg_index_prepare")

    def graph(self):
        inf = self.info()
        adj = torch.empty((inf["n"], inf["R"]), dtype=torch.int32, device="cuda")
        deg = torch.empty(inf["n"], dtype=torch.int32, device="cuda")
        _check(lib().nsg_index_graph(self.h, _ptr(adj), _ptr(deg), _stream()), "nsg_index_graph")
        return adj, deg

    def search(self, queries, k, L):
        queries = _dev(queries, torch.float32)
        nq = queries.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        _check(lib().nsg_search(self.h, _ptr(queries), nq, k, L, _ptr(ids), _ptr(d2), _stream()),
               "nsg_search")
        return ids, d2

    def search_ex(self, queries, k, L, params=None, out=None, counters=True):
        queries = _dev(queries, torch.float32)
        nq = queries.shape[0]
        dev = queries.device
        if out is None:
            out = dict(ids=torch.empty((nq, k), dtype=torch.int32, device=dev),
                       d2=torch.empty((nq, k), dtype=torch.float32, device=dev))
            if counters:
                out.update(n_expand=torch.empty(nq, dtype=torch.int32, device=dev),
                           n_dist=torch.empty(nq, dtype=torch.int32, device=dev),
                           status=torch.empty(nq, dtype=torch.int32, device=dev))
        p = params if params is not None else SearchParams(0, 0, PREC_F32, 0)
        _check(lib().nsg_search_ex(self.h, _ptr(queries), nq, k, L, C.byref(p), _ptr(out["ids"]),
                                   _ptr(out.get("d2")), _ptr(out.get("n_expand")), _ptr(out.get("n_dist")),
                                   _ptr(out.get("status")), _stream()), "nsg_search_ex")
        return out

    def search_host(self, queries, k, L, params=None, ids=None, d2=None):
        """nsg_search_ex on host tensors (page-locked for copy/compute
        overlap): queries [nq][d] float32 in; ids [nq][k] int32 and d2
        (optional) out.  Returns when the results are in host memory."""
        queries = _host(queries, torch.float32)
        nq = queries.shape[0]
        pin = queries.is_pinned()
        ids = torch.empty((nq, k), dtype=torch.int32, pin_memory=pin) if ids is None else _host(ids, torch.int32)
        if d2 is not None:
            d2 = _host(d2, torch.float32)
        p = params if params is not None else SearchParams(0, 0, PREC_F32, 0)
        _check(lib().nsg_search_host(self.h, _ptr(queries), nq, k, L, C.byref(p), _ptr(ids), _ptr(d2),
                                     _stream()), "nsg_search_host")
        return dict(ids=ids, d2=d2)

    def search_partitioned(self, queries, k, L, params=None, out=None):
        """Partition-and-merge search on an index from nsg_build_partitioned:
        every query on every subset, merged to the k smallest (d2, row id)."""
        queries = _dev(queries, torch.float32)
        nq = queries.shape[0]
        dev = queries.device
        if out is None:
            out = dict(ids=torch.empty((nq, k), dtype=torch.int32, device=dev),
                       d2=torch.empty((nq, k), dtype=torch.float32, device=dev))
        p = params if params is not None else SearchParams()
        _check(lib().nsg_search_partitioned(self.h, _ptr(queries), nq, k, L, C.byref(p), _ptr(out["ids"]),
                                            _ptr(out["d2"]), _stream()), "nsg_search_partitioned")
        return out

    def search_trace(self, queries, k, L, cap, params=None):
        """Fixed-L search recording per-step stop features and change flags."""
        queries = _dev(queries, torch.float32)
        nq = queries.shape[0]
        dev = queries.device
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
        feat = torch.zeros((nq, cap, STOP_FEATURES), dtype=torch.float32, device=dev)
        flag = torch.zeros((nq, cap), dtype=torch.uint8, device=dev)
        steps = torch.empty(nq, dtype=torch.int32, device=dev)
        p = params if params is not None else SearchParams()
        _check(lib().nsg_search_trace(self.h, _ptr(queries), nq, k, L, C.byref(p), _ptr(ids), _ptr(feat),
                                      _ptr(flag), _ptr(steps), cap, _stream()), "nsg_search_trace")
        return dict(ids=ids, feat=feat, flag=flag, steps=steps)

    def search_batched(self, queries, k, L, kmax=None, Lmax=None, params=None):
        """Uneven batch: per-query k (int32 [nq]) and L (int32 [nq]) in one
        persistent launch.  Returns ids [nq][kmax], d2, status."""
        queries = _dev(queries, torch.float32)
        k, L = _dev(k, torch.int32), _dev(L, torch.int32)
        nq = queries.shape[0]
        kmax = int(k.max().item()) if kmax is None else kmax
        Lmax = int(L.max().item()) if Lmax is None else Lmax
        dev = queries.device
        ids = torch.empty((nq, kmax), dtype=torch.int32, device=dev)
        d2 = torch.empty((nq, kmax), dtype=torch.float32, device=dev)
        st = torch.empty(nq, dtype=torch.int32, device=dev)
        p = params if params is not None else SearchParams()
        _check(lib().nsg_search_batched(self.h, _ptr(queries), nq, _ptr(k), _ptr(L), kmax, Lmax, C.byref(p),
                                        _ptr(ids), _ptr(d2), _ptr(st), _stream()), "nsg_search_batched")
        return dict(ids=ids, d2=d2, status=st)

    def plan(self, queries, k, L, kmax=None, Lmax=None, params=None, autotune=True):
        return Plan(self, queries, k, L, kmax, Lmax, params, autotune)

    def save(self, path):
        _check(lib().nsg_save(self.h, path.encode()), "nsg_save")


class PlanInfo(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("hash_slots", C.c_int32), ("n_tried", C.c_int32),
                ("best_ms", C.c_float), ("worst_ms", C.c_float), ("warps_per_query", C.c_int32),
                ("pool", C.c_int32), ("stage_rows", C.c_int32)]


class Plan:
    """A bound, autotuned, graph-captured batched search (nsg_plan_*).  The
    tensors passed in stay bound: change their contents, then run()."""

    def __init__(self, index, queries, k, L, kmax, Lmax, params, autotune):
        self.index = index  # keep the index alive
        self.queries = _dev(queries, torch.float32)
        self.k, self.L = _dev(k, torch.int32), _dev(L, torch.int32)
        nq = self.queries.shape[0]
        self.kmax = int(self.k.max().item()) if kmax is None else kmax
        Lmax = int(self.L.max().item()) if Lmax is None else Lmax
        dev = self.queries.device
        self.ids = torch.empty((nq, self.kmax), dtype=torch.int32, device=dev)
        self.d2 = torch.empty((nq, self.kmax), dtype=torch.float32, device=dev)
        self.status = torch.empty(nq, dtype=torch.int32, device=dev)
        self.params = params if params is not None else SearchParams()
        self.h = C.c_void_p()
        _check(lib().nsg_plan_create(index.h, _ptr(self.queries), nq, _ptr(self.k), _ptr(self.L), self.kmax, Lmax,
                                     C.byref(self.params), _ptr(self.ids), _ptr(self.d2), _ptr(self.status),
                                     1 if autotune else 0, _stream(), C.byref(self.h)), "nsg_plan_create")

    def run(self):
        _check(lib().nsg_plan_run(self.h, _stream()), "nsg_plan_run")
        return self.ids, self.d2

    def info(self):
        inf = PlanInfo()
        _check(lib().nsg_plan_info(self.h, C.byref(inf)), "nsg_plan_info")
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def __del__(self):
        try:
            if self.h:
                lib().nsg_plan_free(self.h)
        except Exception:
            pass


def nsg_knn_nndescent(base, K, params=None, with_d2=True):
    """Approximate kNN graph by nn-descent.  Returns (ids, d2 or None,
    iterations run, updates of the last iteration)."""
    base = _dev(base, torch.float32)
    n, d = base.shape
    ids = torch.empty((n, K), dtype=torch.int32, device=base.device)
    d2 = torch.empty((n, K), dtype=torch.float32, device=base.device) if with_d2 else None
    p = params if params is not None else NnDescentParams()
    it, upd = C.c_int32(0), C.c_int64(0)
    _check(lib().nsg_knn_nndescent(_ptr(base), n, d, K, C.byref(p), _ptr(ids), _ptr(d2), C.byref(it),
                                   C.byref(upd), _stream()), "nsg_knn_nndescent")
    return ids, d2, it.value, upd.value


def nsg_build_ex(base, K, L, R, Cap, seed=0, knn_params=None):
    """nsg_build with the kNN stage by nn-descent when knn_params is given."""
    base = _dev(base, torch.float32)
    n, d = base.shape
    h = C.c_void_p()
    kp = C.byref(knn_params) if knn_params is not None else None
    _check(lib().nsg_build_ex(_ptr(base), n, d, K, L, R, Cap, seed, kp, _stream(), C.byref(h)), "nsg_build_ex")
    return Index(h)


def nsg_build_naive(base, K, R, seed=0):
    """NSG-Naive: MRNG selection over the kNN graph's edges (no navigating
    node, no connectivity pass); search it with SearchParams(init_random=...)."""
    base = _dev(base, torch.float32)
    n, d = base.shape
    h = C.c_void_p()
    _check(lib().nsg_build_naive(_ptr(base), n, d, K, R, seed, _stream(), C.byref(h)), "nsg_build_naive")
    return Index(h)


def nsg_build(base, K, L, R, Cap, seed=0):
    base = _dev(base, torch.float32)
    n, d = base.shape
    h = C.c_void_p()
    _check(lib().nsg_build(_ptr(base), n, d, K, L, R, Cap, seed, _stream(), C.byref(h)), "nsg_build")
    return Index(h)


def nsg_build_partitioned(base, part, K, L, R, Cap, seed=0):
    """Partition-and-merge index: one Alg. 2 build per subset (part: host
    int32 [n] subset ids 0..P-1, P = max + 1)."""
    import numpy as np

    base = _dev(base, torch.float32)
    n, d = base.shape
    part = np.ascontiguousarray(np.asarray(part, dtype=np.int32))
    if part.shape != (n,):
        raise ValueError("part needs one subset id per base row")
    h = C.c_void_p()
    _check(lib().nsg_build_partitioned(_ptr(base), n, d, part.ctypes.data_as(C.c_void_p), int(part.max()) + 1,
                                       K, L, R, Cap, seed, _stream(), C.byref(h)), "nsg_build_partitioned")
    return Index(h)


def nsg_index_from_graph(base, adj, nav, deg=None):
    base, adj = _dev(base, torch.float32), _dev(adj, torch.int32)
    n, d = base.shape
    h = C.c_void_p()
    _check(lib().nsg_index_from_graph(_ptr(base), n, d, _ptr(adj), _ptr(deg), adj.shape[1], int(nav),
                                      _stream(), C.byref(h)), "nsg_index_from_graph")
    return Index(h)


def nsg_stop_train(trace, iters=300, lr=1e-2, seed=1, master=None):
    """Train the early-termination MLP on a trace (dict from Index.search_trace).
    Returns (fp16 model tensor [641], fp32 master [641], loss per iteration)."""
    feat, flag, steps = trace["feat"], trace["flag"], trace["steps"]
    nq, cap = flag.shape
    dev = feat.device
    if master is None:
        master = torch.zeros(STOP_PARAMS, dtype=torch.float32, device=dev)
    model = torch.empty(STOP_PARAMS, dtype=torch.float16, device=dev)
    loss = torch.empty(iters, dtype=torch.float32, device=dev)
    _check(lib().nsg_stop_train(_ptr(feat), _ptr(flag), _ptr(steps), nq, cap, iters, lr, seed, _ptr(master),
                                _ptr(model), _ptr(loss), _stream()), "nsg_stop_train")
    return model, master, loss


def nsg_load(path):
    h = C.c_void_p()
    _check(lib().nsg_load(path.encode(), _stream(), C.byref(h)), "nsg_load")
    return Index(h)
