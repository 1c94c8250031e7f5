#!/usr/bin/env python
"""Throughput of NSG search on one GB300: queries/s at recall@10 >= 0.95.

Workload: the SIFT-shaped synthetic set (1,000,000 x 128 integer values 0..255
from a 100-component Gaussian mixture, 10,000 queries), index built with the
paper's Alg. 2 at K=100, L=40, R=50, C=500.  The pool size L is swept over
100, 125, ..., 400 and 500..1000 (k=100), and between the last grid point
below a recall target and the first one above it the smallest integer L
reaching the target is found by bisection; the reported point is the
highest-QPS L whose mean recall@10 (Eq. 1, against the exact ground truth)
is >= 0.95.

Forms: plain (FP32 traversal, exactly Alg. 1), the precision forms (BF16 or
FP8-e4m3 traversal distances with FP32 accumulation, or an 8-bit copy with
exact int32 sums; FP32 re-rank of the final pool when the copy is lossy),
and the learned-stop forms (an MLP trained on the GPU from search traces of
a separate query batch ends each search early; swept over its probability
threshold).  On this integer workload the BF16 and U8 copies are exact, so
those forms return the plain form's results bit for bit.  `value` is the form with the highest QPS
at recall@10 >= 0.95 ("chosen"); `plain` holds the plain form beside it.

A step = one nsg_search_ex launch over the whole 10,000-query batch, inputs
resident in HBM.  The base (512 MB) is larger than L2 (129 MB).
`e2e` repeats the step through the C ABI's host-buffer call (nsg_search_host)
on page-locked host memory: host->device copy of the queries, search,
device->host copy of the ids, all inside the call.

`configs` (the default SIFT-shaped run at N = 1): the GIST-shaped precision
configuration (1M x 960 float, 1,000 queries: plain, BF16, FP8, U8 forms) and
the DEEP-shaped batched one (10M x 96 unit vectors, 100,000 uneven queries in
one autotuned, graph-replayed launch; the 8-bit form's learned stop trained on
this index's traces), each a `--compact` run of this script in a child
process (its own short L grid), summarised.

Multi-GPU: queries are independent, so each rank searches its own batch on
its own replica of the index (weak scaling, no collective on the data path).

CPU baseline (`cpu_baseline`, and `--impl reference`): the CPU oracle's
Alg. 1 (Section 3.6), single-threaded and on all host cores, searching the
same index at the same pool size on bounded query samples.  The index is the
library's build: the oracle needs hours of host time to build a 1M-row index
(its kNN stage alone is an O(n^2 d) serial scan), and the library's build
equals the oracle's wherever the tests compare them.  The oracle's exact
serial scan (the paper's own baseline, Section 4.1.2) is reported beside it.

--profile-case search|knn|build runs one small kernel family for a profiler
(see `profile_case`) and prints one line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/sec at recall@10=0.95 on 1 GB300, chosen vs plain form; % HBM peak"
UNIT = "queries/s"
TARGET = 0.95
# Per workload: build parameters, the L grid, result size k, and a description.
# `sift` is the headline configuration; `gist` (float, d=960) and `deep`
# (10M x 96 unit vectors) are the precision and batched configurations;
# `rand4m` and `gauss5m` are the paper's own high-LID synthetic sets.
WORKLOADS = {
    # L 100..400 is the sweep of the SIFT-shaped configuration; 500..1000 reach recall@10 = 0.99
    "sift": dict(build=dict(K=100, L=40, R=50, C=500), L_grid=list(range(100, 401, 25)) + [500, 600, 800, 1000], k=100,
                 desc="sift-shaped 1,000,000 x 128 int 0..255 GMM(100), 10,000 queries", integer=True),
    "gist": dict(build=dict(K=100, L=60, R=70, C=500),
                 L_grid=[10, 20, 40, 60, 80, 100, 150, 200, 300, 400, 500, 1000, 2000, 4000],
                 compact_grid=[100, 200, 300, 400, 600, 1000, 2000], compact_forms=("bf16", "fp8", "u8"),
                 k=100, desc="gist-shaped 1,000,000 x 960 f32 [0,1] GMM(50), 1,000 queries"),
    # the kNN stage by nn-descent (16 samples, 16 reverse, 12 iterations), as the
    # paper builds its million-scale kNN graphs (Section 3.6): on this tight
    # 1,000-cluster mixture the exact graph links mostly within clusters
    "deep": dict(build=dict(K=64, L=60, R=32, C=500), knn=(16, 16, 12),
                 L_grid=[20, 40, 60, 100, 150, 200, 300, 400, 500, 700, 1000, 2000, 4000],
                 compact_grid=[200, 400, 700, 1000], compact_forms=("u8",), compact_stop=("u8",),
                 k=100, desc="deep-shaped 10,000,000 x 96 f32 unit-norm GMM(1000), 100,000 queries"),
    # the paper's own synthetic sets (Table 1); R = 220 is the maximum out-degree it reports for them
    "rand4m": dict(build=dict(K=100, L=60, R=220, C=500),
                   L_grid=[20, 40, 60, 100, 150, 200, 300, 400, 500, 700, 1000, 2000, 4000],
                   k=100, desc="RAND4M: 4,000,000 x 128 i.i.d. U(0,1), 10,000 queries"),
    "gauss5m": dict(build=dict(K=100, L=60, R=220, C=500),
                    L_grid=[20, 40, 60, 100, 150, 200, 300, 400, 500, 700, 1000, 2000, 4000],
                    k=100, desc="GAUSS5M: 5,000,000 x 128 i.i.d. N(0,3), 10,000 queries"),
}
STOP_TRACE_LS, STOP_TRACE_CAP, STOP_ITERS = (100, 200, 400), 1024, 300
STOP_THRESHOLDS = [0.9, 0.95, 0.98]
RECALL_TARGETS = (0.95, 0.99)
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sift", choices=sorted(WORKLOADS))
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    p.add_argument("--naive", action="store_true", help="also build and sweep NSG-Naive (ablation)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the partition-and-merge and nn-descent legs")
    p.add_argument("--compact", action="store_true",
                   help="the workload's own forms on a short L grid, learned stop only where the workload "
                        "names it (a configuration run)")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the GIST- and DEEP-shaped configuration runs the default SIFT-shaped line carries")
    p.add_argument("--profile-case", choices=["search", "knn", "build", "nndescent", "partitioned"], default=None,
                   help="run one kernel family on a small SIFT-shaped case for a profiler")
    p.add_argument("--n", type=int, default=300000, help="--profile-case: base rows")
    p.add_argument("--nq", type=int, default=2000, help="--profile-case: queries")
    p.add_argument("--L", type=int, default=150, help="--profile-case search: pool size")
    p.add_argument("--K", type=int, default=100, help="--profile-case knn: neighbours per row")
    p.add_argument("--prec", type=int, default=0, help="--profile-case search: 0 FP32, 1 BF16, 2 FP8, 3 U8")
    p.add_argument("--wpq", type=int, default=1, help="--profile-case search: warps per query (0: the library's)")
    p.add_argument("--reps", type=int, default=2, help="--profile-case search: launches")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank values over the process group (the
    slowest rank sets a step's time); the values unchanged on one process."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_qps(world, nq, ms):
    """Whole-job queries/s: every rank searches its own nq queries per step."""
    return world * nq / (ms / 1e3)


def rank_query_seed(rank, base_seed):
    """Each rank draws its own query batch (weak scaling); the base is shared."""
    return base_seed + 1000 * rank


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows, self.proc = [], None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        return self.summarize(self.rows)

    @staticmethod
    def summarize(rows):
        """Median SM clock, the maximum clock and the throttle reasons seen
        active in rows of the query fields (split on commas)."""
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9
                          for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


SEARCH_SOURCES = ("common.cuh", "search_core.cuh", "lowp.cuh", "stage.cuh", "search_kern.cuh", "search.cu")
PRUNE_SOURCES = ("common.cuh", "search_core.cuh", "build.cu")


def refine_L(pts, t, recall_at, qps_at):
    """Smallest integer L between the last sweep point below recall t and the
    first one at or above it that still reaches t (bisection, recall growing
    with L), as a new sweep point; None when no L below that grid point does
    or no grid point reaches t.  recall_at(L) and qps_at(L) measure one L."""
    pts = sorted(pts, key=lambda p: p["L"])
    above = [i for i, p in enumerate(pts) if p["recall10"] >= t]
    if not above or above[0] == 0:
        return None
    lo, hi, hi_rec = pts[above[0] - 1]["L"], pts[above[0]]["L"], pts[above[0]]["recall10"]
    grid_hi = hi
    while hi - lo > 1:
        mid = (lo + hi) // 2
        r = recall_at(mid)
        if r >= t:
            hi, hi_rec = mid, r
        else:
            lo = mid
    if hi == grid_hi:
        return None
    return {"L": hi, "recall10": hi_rec, "qps": qps_at(hi), "refined": True}


def kernel_source_hash(files=SEARCH_SOURCES):
    """Hash of a kernel's code with comments and blank lines removed, so that
    the hash changes with the code and not with its documentation."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1707_00143_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in src.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one
# search launch, per query, keyed by (kernel source hash, workload, form, L):
# profiles/search_kernel_u8_sift.md has the capture.  A source change changes
# the hash, and `traffic` is null until re-measured.
NCU_TRAFFIC = {
    ("fc53c47ea7d2373f", "sift", "u8", 138): (1_167_627_264 + 15_439_104) / 10_000,
}
# warp instructions of one search launch, per query (smsp__inst_executed.sum of the
# same capture command with that metric), keyed like NCU_TRAFFIC: the issue roofline
NCU_INSTRUCTIONS = {
    ("fc53c47ea7d2373f", "sift", "u8", 138): 1_369_312_578 / 10_000,
}
# the same for the MRNG edge selection of the build, per node, keyed by
# (source hash, workload): profiles/prune_kernel_sift1m.md
PRUNE_TRAFFIC = {
    ("4744460958126e69", "sift"): (18_545_727_232 + 135_220_736 + 16_066_647_040 + 114_126_592) / 1_000_000,
}


def bench_config(W, world, base):
    """The workload a line measures: the same dict in both arms."""
    knn = "exact (tensor-core scan)" if "knn" not in W else "nn-descent (samples %d, reverse %d, iterations %d)" % W["knn"]
    return {"workload": W["desc"], "build": W["build"], "knn_stage": knn, "k": W["k"], "target_recall10": TARGET,
            "parallelism": f"replicas{world}", "l2": f"inputs larger than L2 ({base.nbytes >> 20} MB base)"}


def build_index(capi, bt, W, seed=0):
    """Alg. 2 on the workload's kNN stage: exact, or nn-descent where W names one."""
    B = W["build"]
    if "knn" in W:
        return capi.nsg_build_ex(bt, B["K"], B["L"], B["R"], B["C"], seed=seed,
                                 knn_params=capi.NnDescentParams(*W["knn"], 0.001, 1))
    return capi.nsg_build(bt, B["K"], B["L"], B["R"], B["C"], seed=seed)


def _timed_sample(fn, q, per_q_budget, cap):
    """Run fn on the first m queries, m sized from a 16-query probe so the
    call takes about `per_q_budget` seconds; returns (m, seconds)."""
    t = time.perf_counter()
    fn(q[:16])
    per_q = max((time.perf_counter() - t) / 16, 1e-7)
    m = int(max(16, min(cap, len(q), per_q_budget / per_q)))
    t = time.perf_counter()
    fn(q[:m])
    return m, time.perf_counter() - t


def cpu_serial_scan(base, q, budget_s=5.0):
    """Oracle serial scan (exact kNN: recall 1.0) on a bounded query sample."""
    import oracle

    cores = os.cpu_count() or 1
    m, el = _timed_sample(lambda qs: oracle.knn_query(base, qs, 10, nthreads=cores), q, budget_s, len(q))
    return {"value": m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"serial scan (exact kNN, recall@10 = 1.0) of the first {m} queries against "
                      f"the full {len(base)}-row base, {cores} host threads"}


def cpu_alg1(adj, deg, base, nav, q, k, L, budget_s=8.0):
    """The oracle's Alg. 1 (plain, single-threaded per query) on the given
    index at pool size L: one sample on one host thread (queries/s per core)
    and one on every host thread (disjoint query ranges)."""
    import oracle

    cores = os.cpu_count() or 1

    counts = {}

    def run(qs, nt):
        _, _, ne, nd = oracle.search(adj, base, nav, qs, k, L, deg=deg, nthreads=nt)
        counts["n_expand"], counts["n_dist"] = ne, nd

    m1, el1 = _timed_sample(lambda qs: run(qs, 1), q, budget_s / 2, 2000)
    m, el = _timed_sample(lambda qs: run(qs, cores), q, budget_s, len(q))
    out = {"value": m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"oracle Alg. 1 (k = {k}, L = {L}) over the first {m} queries on {cores} host threads, "
                     f"on the index the library built",
           "single_thread": {"value": m1 / el1, "queries": m1}}
    return out, counts


def profile_case(args):
    """One kernel family on a small case of --workload (SIFT-shaped by
    default), for a profiler: `search` builds an index (the workload's build
    parameters; SIFT-shaped K=100, L=40, R=50, C=500) on an n-row base and runs
    `--reps` searches of nq queries (top 100, pool --L) in the precision form
    --prec with --wpq warps per query; `knn` runs one brute-force kNN graph
    (K = --K); `build` one index construction; `nndescent` one nn-descent
    kNN graph (K = --K, 16 samples and 16 reverse samples, 12 iterations);
    `partitioned` a 4-subset partitioned index and `--reps` partitioned
    searches (top 100, pool --L)."""
    import torch

    from paper_1707_00143_gb300 import build as nsg_build_mod
    from paper_1707_00143_gb300 import capi, datagen

    nsg_build_mod.build()
    torch.cuda.set_device(0)
    base, q = datagen.workload(args.workload, n=args.n, nq=args.nq)
    bt, qt = torch.from_numpy(base).cuda(), torch.from_numpy(q).cuda()
    B = WORKLOADS[args.workload]["build"]
    if args.profile_case == "knn":
        capi.nsg_knn_init(bt, args.K, with_d2=False)
        torch.cuda.synchronize()
        print(f"knn n={args.n} K={args.K} done")
        return
    if args.profile_case == "nndescent":
        _, _, it, upd = capi.nsg_knn_nndescent(bt, args.K, capi.NnDescentParams(16, 16, 12, 0.001, 1), with_d2=False)
        torch.cuda.synchronize()
        print(f"nndescent n={args.n} K={args.K} iterations={it} last_updates={upd} done")
        return
    if args.profile_case == "partitioned":
        pidx = capi.nsg_build_partitioned(bt, datagen.even_partition(args.n, 4, seed=17), 100, 40, 50, 500)
        if args.prec:
            pidx.prepare(args.prec)
        prm = capi.SearchParams(0, 0, args.prec, 0, -1)
        for _ in range(args.reps):
            pidx.search_partitioned(qt, 100, args.L, params=prm)
        torch.cuda.synchronize()
        print(f"partitioned n={args.n} nq={args.nq} L={args.L} prec={args.prec} done")
        return
    idx = build_index(capi, bt, WORKLOADS[args.workload])
    if args.profile_case == "build":
        torch.cuda.synchronize()
        print(f"build n={args.n} done: {idx.info()}")
        return
    if args.prec:
        idx.prepare(args.prec)
    prm = capi.SearchParams(0, 0, args.prec, 0, -1, None, 0.5, 0, 0, 0, 0, args.wpq)
    for _ in range(args.reps):
        idx.search_ex(qt, 100, args.L, params=prm, counters=False)
    torch.cuda.synchronize()
    print(f"search n={args.n} nq={args.nq} L={args.L} prec={args.prec} wpq={args.wpq} done")


def run_reference(args):
    """The oracle's Alg. 1 on the workload's index, at the smallest pool size
    whose recall@10 on a 1,000-query sample reaches the target (the sweep
    and bisection of this arm, with the oracle's exact serial scan as ground
    truth); each step searches a sample of queries on every host thread."""
    world, rank, local = dist_env()
    if rank != 0:
        return
    import numpy as np
    import torch

    from paper_1707_00143_gb300 import build as nsg_build_mod
    from paper_1707_00143_gb300 import capi, datagen
    import oracle

    oracle.compile_lib()
    W = WORKLOADS[args.workload]
    B = W["build"]
    base, q = datagen.workload(args.workload)
    cores = os.cpu_count() or 1
    # the index (setup, untimed): the library's build, equal to the oracle's own
    nsg_build_mod.build()
    torch.cuda.set_device(local)
    idx = build_index(capi, torch.from_numpy(base).cuda(), W, seed=0)
    adj, deg = (t.cpu().numpy() for t in idx.graph())
    nav = idx.info()["nav"]
    del idx
    torch.cuda.empty_cache()
    # operating point: recall@10 of the oracle's own results on a query sample
    ns = min(1000, len(q))
    gt, _ = oracle.knn_query(base, q[:ns], 10, nthreads=cores)

    def recall_at(L):
        ids, _, _, _ = oracle.search(adj, base, nav, q[:ns], 10, L, deg=deg, nthreads=cores)
        return oracle.recall(ids, gt, 10)

    pts = []
    for L in W["L_grid"]:
        pts.append({"L": L, "recall10": recall_at(L)})
        if pts[-1]["recall10"] >= TARGET:
            break
    p = refine_L(pts, TARGET, recall_at, lambda L: None)
    ok = [x for x in pts if x["recall10"] >= TARGET]
    L = p["L"] if p else (ok[0]["L"] if ok else W["L_grid"][-1])
    rec = p["recall10"] if p else (ok[0]["recall10"] if ok else pts[-1]["recall10"])
    kq = min(W["k"], L)
    m = 2000
    times = []
    for s in range(args.warmup + args.steps):
        lo = (s * m) % len(q)
        qs = q[lo:lo + m]
        t = time.perf_counter()
        oracle.search(adj, base, nav, qs, kq, L, deg=deg, nthreads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    v = len(qs) / (ms / 1e3)
    t = time.perf_counter()
    oracle.search(adj, base, nav, q[:200], kq, L, deg=deg, nthreads=1)
    single = 200 / (time.perf_counter() - t)
    sample = (f"oracle Alg. 1 (k = {kq}, L = {L}) over {m} queries per step on {cores} host threads, "
              f"on the index the library built")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(W, 1, base),
        "operating_point": {"form": "oracle Alg. 1 (FP32)", "L": L, "recall10_sample": rec,
                            "sample_queries": ns, "sweep": pts},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": single, "queries": 200}},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def sweep_point(L_grid, run_recall, run_ms, nq, target=TARGET):
    """Grid sweep + bisection to the smallest L reaching `target`; returns
    (point with L, recall10, qps | None, sweep points)."""
    pts = []
    for L in L_grid:
        pts.append({"L": L, "recall10": run_recall(L), "qps": nq / (run_ms(L) / 1e3)})
        if pts[-1]["recall10"] >= target:
            break
    p = refine_L(pts, target, run_recall, lambda L: nq / (run_ms(L) / 1e3))
    if p is not None:
        pts.append(p)
        pts.sort(key=lambda x: x["L"])
    ok = [x for x in pts if x["recall10"] >= target]
    return (max(ok, key=lambda x: x["qps"]) if ok else None), pts


def extra_legs(capi, datagen, bt, qt, gt, base, W, forms, chosen_form, nq, kq, recall10, ev0, ev1, st, args):
    """Partition-and-merge search (Sections 4.2, 4.3) at P = 4 and 8 subsets and
    a build whose kNN stage is nn-descent (Sec. 3.5 (ii)): build seconds and
    queries/s at recall@10 >= 0.95 in the chosen precision form."""
    import torch

    B = W["build"]
    prec = forms[chosen_form.split("+")[0]].precision
    out = {}

    def timer(fn, reps=2):
        fn()
        ev0.record(st)
        for _ in range(reps):
            fn()
        ev1.record(st)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / reps

    parts = {}
    for P in (4, 8):
        part = datagen.even_partition(len(base), P, seed=17)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pidx = capi.nsg_build_partitioned(bt, part, B["K"], B["L"], B["R"], B["C"], seed=0)
        torch.cuda.synchronize()
        b_s = time.perf_counter() - t0
        if prec:
            pidx.prepare(prec)
        prm = capi.SearchParams(0, 0, prec, 0, -1)
        bufs = {}

        def res(L):
            k = kq(L)
            if k not in bufs:
                bufs[k] = pidx.search_partitioned(qt, k, L, params=prm)
            return pidx.search_partitioned(qt, k, L, params=prm, out=bufs[k])

        best, pts = sweep_point(W["L_grid"], lambda L: recall10(res(L)), lambda L: timer(lambda: res(L)), nq)
        info = pidx.info()
        parts[str(P)] = {"build_seconds": b_s, "build_ms_sum_of_subsets": {k: info[k] for k in (
            "ms_knn", "ms_collect", "ms_prune", "ms_connect")}, "at_recall10_0.95": best, "sweep": pts}
        del pidx
    out["partitioned"] = {"form": chosen_form.split("+")[0], "partition": "even random (seed 17)", "P": parts}

    nnd = capi.NnDescentParams(16, 16, 12, 0.001, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nidx = capi.nsg_build_ex(bt, B["K"], B["L"], B["R"], B["C"], seed=0, knn_params=nnd)
    torch.cuda.synchronize()
    b_s = time.perf_counter() - t0
    ninfo = nidx.info()
    # graph recall of the nn-descent kNN stage against the exact one, on sampled rows
    rows = torch.arange(0, len(base), max(1, len(base) // 2000), device=bt.device)
    ex_ids, _ = capi.nsg_knn_query(bt, bt[rows].contiguous(), B["K"] + 1)
    nn_ids, _, _, _ = capi.nsg_knn_nndescent(bt, B["K"], nnd, with_d2=False)
    ex_h, nn_h, rows_h = ex_ids.cpu().numpy(), nn_ids[rows].cpu().numpy(), rows.cpu().numpy()
    g_rec = sum(len(set(nn_h[i]) & (set(ex_h[i]) - {int(rows_h[i])})) for i in range(len(rows_h))) / (
        B["K"] * len(rows_h))
    if prec:
        nidx.prepare(prec)
    prm = capi.SearchParams(0, 0, prec, 0, -1)
    bufs = {}

    def nres(L):
        k = kq(L)
        o = nidx.search_ex(qt, k, L, params=prm, out=bufs.get(k), counters=False)
        bufs[k] = o
        return o

    best, pts = sweep_point(W["L_grid"], lambda L: recall10(nres(L)), lambda L: timer(lambda: nres(L)), nq)
    out["nndescent"] = {"params": {"sample": 16, "reverse": 16, "iters": 12, "delta": 0.001},
                        "iterations": ninfo["knn_iters"], "build_seconds": b_s,
                        "build_ms": {k: ninfo[k] for k in ("ms_knn", "ms_collect", "ms_prune", "ms_connect",
                                                            "ms_total")},
                        "knn_graph_recall_vs_exact": g_rec, "graph_recall_rows": int(len(rows_h)),
                        "form": chosen_form.split("+")[0], "at_recall10_0.95": best, "sweep": pts}
    del nidx
    return out


def ground_truth(capi, bt, qt, W, k=10):
    """Exact k nearest base rows of every query: the tensor-core kNN on
    integer data (exact there), the FP32 CUDA-core scan otherwise (the
    tensor-core path ranks float data by BF16 products before its FP32
    re-rank, which can miss a true neighbour)."""
    if W.get("integer"):
        return capi.nsg_knn_query(bt, qt, k)
    old = os.environ.get("NSG_KNN_ENGINE")
    os.environ["NSG_KNN_ENGINE"] = "scan"
    try:
        return capi.nsg_knn_query(bt, qt, k)
    finally:
        if old is None:
            del os.environ["NSG_KNN_ENGINE"]
        else:
            os.environ["NSG_KNN_ENGINE"] = old


# The configurations the default SIFT-shaped line carries besides its own: the
# GIST-shaped precision forms (1M x 960, 1,000 queries) and the DEEP-shaped
# batched uneven queries (10M x 96, 100,000 queries), each a compact run of
# this script in a child process, with a time limit in seconds.
CONFIG_RUNS = (("gist", 360), ("deep", 480))
CONFIG_KEYS = ("metric", "value", "unit", "ms_per_step", "dtype", "config", "operating_point", "plain",
               "chosen_over_plain", "roofline", "e2e", "clocks", "gpu_launches", "build_seconds", "build_ms", "index",
               "batched", "precision_error_vs_fp64", "learned_stop")


def config_runs(args):
    out = {}
    for wl, limit in CONFIG_RUNS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", wl, "--compact", "--no-extras", "--no-cpu",
               "--steps", str(args.steps), "--warmup", str(args.warmup)]
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=limit)
        except subprocess.TimeoutExpired:
            out[wl] = {"error": "no result within %d s" % limit}
            continue
        lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
        if r.returncode != 0 or not lines:
            tail = (r.stderr.strip().splitlines() or ["?"])[-1]
            out[wl] = {"error": "exit %d: %s" % (r.returncode, tail[:300])}
            continue
        d = json.loads(lines[-1])
        res = {k: d.get(k) for k in CONFIG_KEYS}
        res["at_recall10"] = {t: {f: ({"L": v["L"], "qps": v["qps"]} if v else None)
                                  for f, v in d["at_recall10"][t]["best"].items()} for t in d.get("at_recall10", {})}
        res["stop_vs_fixed_L"] = {t: d["at_recall10"][t].get("stop_vs_fixed_L") for t in d.get("at_recall10", {})}
        res["command"] = " ".join(["python", "bench.py"] + cmd[2:])
        res["seconds"] = time.perf_counter() - t0
        out[wl] = res
    return out


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1707_00143_gb300 import build as nsg_build_mod
    from paper_1707_00143_gb300 import capi, datagen

    if rank == 0:
        nsg_build_mod.build()
    if world > 1:
        dist.barrier()
    capi.lib()

    # inputs: same base on every rank (a replica), a distinct query batch per rank
    W = WORKLOADS[args.workload]
    BUILD, L_GRID, K_RESULTS = W["build"], W["L_grid"], W["k"]
    if args.compact:
        L_GRID = W.get("compact_grid", L_GRID)
    base, q = datagen.workload(args.workload, seed_query=rank_query_seed(rank, datagen.SEED_QUERY))
    n, d = base.shape
    nq = len(q)
    bt = torch.from_numpy(base).cuda()
    qt = torch.from_numpy(q).cuda()
    st = torch.cuda.current_stream()

    t0 = time.perf_counter()
    idx = build_index(capi, bt, W, seed=0)
    build_s = time.perf_counter() - t0
    gt, gt_d2 = ground_truth(capi, bt, qt, W)

    # the forms: plain FP32 traversal, and the precision forms (BF16 / FP8-e4m3
    # traversal with FP32 accumulation; FP32 re-rank of the pool when the copy is lossy)
    forms = {"plain": capi.SearchParams(0, 0, capi.PREC_F32, 0)}
    for name, prec in (("bf16", capi.PREC_BF16), ("fp8", capi.PREC_FP8), ("u8", capi.PREC_U8)):
        if args.compact and name not in W.get("compact_forms", (name,)):
            continue
        idx.prepare(prec)
        forms[name] = capi.SearchParams(0, 0, prec, 0, -1)
    train_s, stop_loss = None, None
    stop_bases = W.get("compact_stop", ()) if args.compact else ("plain", "u8")
    if stop_bases:
        # learned early termination: traces of a separate query batch (its own
        # seed, never timed) -> MLP trained on the GPU -> stop rule in the kernel
        _, q_train = datagen.workload(args.workload, n=1, nq=nq, seed_query=datagen.SEED_QUERY + 500 + 1000 * rank)
        t1 = time.perf_counter()
        # traces at three pool sizes (the features are relative to L), one model
        qtr = torch.from_numpy(q_train).cuda()
        parts = [idx.search_trace(qtr[i::len(STOP_TRACE_LS)].contiguous(), 10, Lt, STOP_TRACE_CAP,
                                  params=capi.SearchParams(0, 0, capi.PREC_F32, 0, -1, None, 0.5, 10))
                 for i, Lt in enumerate(STOP_TRACE_LS)]
        trace = {key: torch.cat([t[key] for t in parts]) for key in ("feat", "flag", "steps")}
        del parts
        stop_model, _, stop_loss = capi.nsg_stop_train(trace, iters=STOP_ITERS, lr=1e-2, seed=1)
        del trace
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        for th in STOP_THRESHOLDS:
            for base_name in stop_bases:
                b = forms[base_name]
                forms[f"{base_name}+stop{th}"] = capi.SearchParams(0, 0, b.precision, 0, -1, stop_model, th, 10)
    info = idx.info()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    outs = {}  # output buffers per result size

    def kq(L):  # results per query at pool size L (k <= L; recall@10 needs 10)
        return min(K_RESULTS, L)

    def run(L, params):
        o = idx.search_ex(qt, kq(L), L, params=params, out=outs.get(kq(L)), counters=False)
        outs[kq(L)] = o
        return o

    def timed(params, L, reps):
        ev0.record(st)
        for _ in range(reps):
            run(L, params)
        ev1.record(st)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / reps

    def recall10(o):
        return capi.nsg_recall(o["ids"][:, :10].contiguous(), gt, 10).sum().item() / (10.0 * nq)

    def refine(pts, prm, t):
        return refine_L(pts, t, lambda L: recall10(run(L, prm)), lambda L: nq / (timed(prm, L, 2) / 1e3))

    # sweep L per form: recall@10 and a quick timing per point, then the
    # smallest L reaching each recall target between two grid points
    sweeps, best = {}, {}
    for name, prm in forms.items():
        pts = []
        for L in L_GRID:
            rec = recall10(run(L, prm))
            ms = timed(prm, L, 2)
            pts.append({"L": L, "recall10": rec, "qps": nq / (ms / 1e3)})
        for t in RECALL_TARGETS:
            p = refine(pts, prm, t)
            if p is not None and all(q["L"] != p["L"] for q in pts):
                pts.append(p)
        pts.sort(key=lambda p: p["L"])
        sweeps[name] = pts
        ok = [p for p in pts if p["recall10"] >= TARGET]
        best[name] = max(ok, key=lambda p: p["qps"]) if ok else None
    cands = {k: v for k, v in best.items() if v is not None}
    at_recall = {}
    for t in RECALL_TARGETS:
        per = {}
        for name, pts in sweeps.items():
            ok = [p for p in pts if p["recall10"] >= t]
            per[name] = max(ok, key=lambda p: p["qps"]) if ok else None
        # each learned-stop form against the fixed-L search of the same precision
        stop_vs_fixed = {name: per[name]["qps"] / per[name.split("+")[0]]["qps"]
                         for name in per if "+stop" in name and per[name] and per[name.split("+")[0]]}
        at_recall[str(t)] = {"best": per, "stop_vs_fixed_L": stop_vs_fixed}
    chosen_form = max(cands, key=lambda k: cands[k]["qps"]) if cands else "plain"
    plain_L = best["plain"]["L"] if best["plain"] else L_GRID[-1]
    L = cands[chosen_form]["L"] if cands else L_GRID[-1]
    prm = forms[chosen_form]

    # traversal-distance error of the precision forms against FP64: search a
    # query sample without re-rank, recompute the returned ids' distances in
    # float64 on the host, compare in the copy's units scaled back
    prec_err = {}
    qs_n = min(200, nq)
    for name, scale in (("bf16", 1.0), ("fp8", info["fp8_scale"]), ("u8", info["u8_scale"])):
        if name not in forms:
            continue
        o = idx.search_ex(qt[:qs_n], 10, L_GRID[len(L_GRID) // 2],
                          params=capi.SearchParams(0, 0, forms[name].precision, 0, 0), counters=False)
        ids_s = o["ids"].cpu().numpy()
        d2_s = o["d2"].cpu().numpy().astype(np.float64) / (scale * scale)
        ex = ((base[ids_s].astype(np.float64) - q[:qs_n, None, :].astype(np.float64)) ** 2).sum(-1)
        rel = np.abs(d2_s - ex) / np.maximum(ex, 1e-30)
        prec_err[name] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                          "queries": qs_n, "k": 10, "exact_copy": bool(info["has_" + name] == 2)}

    # algorithmic bytes at the chosen point: unique distance and expansion counts
    # (the chosen form's parameters, learned stop included, with an exact visited set)
    big = capi.SearchParams.from_buffer_copy(prm)
    big.hash_slots, big.warps_per_cta = 16384, 0
    kc = kq(L)
    cnt = idx.search_ex(qt, kc, L, params=big)
    n_dist = cnt["n_dist"].to(torch.int64).sum().item()
    n_expand = cnt["n_expand"].to(torch.int64).sum().item()
    R = info["R"]
    base_form = chosen_form.split("+")[0]
    row_bytes = {"plain": d * 4, "bf16": ((d + 7) // 8) * 16, "fp8": ((d + 15) // 16) * 16,
                 "u8": ((d + 15) // 16) * 16}[base_form]
    lossy = {"plain": False, "bf16": info["has_bf16"] == 1, "fp8": info["has_fp8"] == 1,
             "u8": info["has_u8"] == 1}[base_form]
    bytes_launch = (n_dist * row_bytes + n_expand * R * 4 + nq * (d * 4 + kc * 8)
                    + (nq * L * d * 4 if lossy else 0))

    # timed region: inputs resident in HBM, one search launch per step
    for _ in range(args.warmup):
        run(L, prm)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    time.sleep(0.4)
    torch.cuda.synchronize()
    ms_step = timed(prm, L, args.steps)
    torch.cuda.synchronize()
    clocks = clk.stop()
    rec_chosen = recall10(outs[kc])
    # tie-aware recall@10: a returned id counts when its distance is within the
    # true 10th distance (integer data has many exact ties)
    rec_chosen_ties = (outs[kc]["d2"][:, :10] <= gt_d2[:, 9:10]).sum().item() / (10.0 * nq)
    ms_plain = timed(forms["plain"], plain_L, args.steps)
    rec_plain = recall10(outs[kq(plain_L)])
    ms_step, ms_plain = max_over_ranks([ms_step, ms_plain], "cuda")
    if world > 1:
        dist.barrier()

    # end to end through the C ABI's host-buffer call (nsg_search_host): the
    # queries are copied in and the ids copied back inside every step
    qh = torch.from_numpy(q).pin_memory()
    ids_h = torch.empty((nq, kc), dtype=torch.int32).pin_memory()
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            e2e_t0 = time.perf_counter()
        idx.search_host(qh, kc, L, params=prm, ids=ids_h)
    e2e_ms = 1e3 * (time.perf_counter() - e2e_t0) / args.steps
    e2e_same = torch.equal(ids_h, run(L, prm)["ids"].cpu())
    e2e_ms = max_over_ranks([e2e_ms], "cuda")[0]

    # NSG-Naive (Section 4.1.2, the paper's ablation): MRNG selection over the
    # kNN graph's edges, no navigating node or connectivity pass, searched by
    # Alg. 1 from L random nodes; the plain form at a few pool sizes
    naive = None
    if args.naive:
        t2 = time.perf_counter()
        nidx = capi.nsg_build_naive(bt, BUILD["K"], BUILD["R"], seed=0)
        torch.cuda.synchronize()
        nb_s = time.perf_counter() - t2
        npts = []
        for Ln in L_GRID[:: max(1, len(L_GRID) // 5)]:
            nprm = capi.SearchParams(0, 0, capi.PREC_F32, 0, -1, None, 0.5, 0, 0, Ln, 1)
            o = nidx.search_ex(qt, kq(Ln), Ln, params=nprm, counters=False)
            torch.cuda.synchronize()
            ev0.record(st)
            for _ in range(2):
                o = nidx.search_ex(qt, kq(Ln), Ln, params=nprm, out=o, counters=False)
            ev1.record(st)
            ev1.synchronize()
            npts.append({"L": Ln, "recall10": recall10(o), "qps": nq / (ev0.elapsed_time(ev1) / 2 / 1e3)})
        ninfo = nidx.info()
        naive = {"build_seconds": nb_s, "avg_degree": ninfo["avg_degree"], "init": "L random nodes",
                 "sweep": npts, "nsg_plain_sweep": sweeps["plain"]}
        del nidx

    # batched uneven queries on the same index: k from {1, 10, 100}, L uniform
    # in 20..500, one autotuned persistent launch replayed as a CUDA graph,
    # against the same batch padded to one fixed (k, L) = (100, 500) launch
    kb, Lb = datagen.uneven_k_L(nq, seed=91 + rank, ks=(1, 10, 100), l_lo=20, l_hi=500)
    kbt, Lbt = torch.from_numpy(kb).cuda(), torch.from_numpy(Lb).cuda()
    bprm = forms[chosen_form.split("+")[0]]
    plan = idx.plan(qt, kbt, Lbt, params=bprm, autotune=True)
    pinfo = plan.info()
    for _ in range(args.warmup):
        plan.run()
    ev0.record(st)
    for _ in range(args.steps):
        plan.run()
    ev1.record(st)
    ev1.synchronize()
    ms_batched = ev0.elapsed_time(ev1) / args.steps
    ms_padded = timed(bprm, int(Lb.max()), max(2, args.steps // 2))
    ms_batched, ms_padded = max_over_ranks([ms_batched, ms_padded], "cuda")
    batched = {"form": chosen_form.split("+")[0], "queries": nq, "k_choices": [1, 10, 100], "L_range": [20, 500],
               "value": job_qps(world, nq, ms_batched), "ms_per_step": ms_batched,
               "padded_k100_L500": {"value": job_qps(world, nq, ms_padded), "ms_per_step": ms_padded},
               "plan": pinfo}

    extras = {} if args.no_extras else extra_legs(capi, datagen, bt, qt, gt, base, W, forms, chosen_form, nq, kq,
                                                   recall10, ev0, ev1, st, args)

    # CPU baseline: the oracle's Alg. 1 on this index; its unique expansion and
    # distance counts are the algorithmic counts of the roofline where it
    # covered the whole batch (the GPU counting pass is checked against them)
    cpu, count_src = None, "GPU counting pass (16,384-slot visited set)"
    counts_check = None
    if rank == 0 and world == 1 and not args.no_cpu:
        adj_h, deg_h = (t.cpu().numpy() for t in idx.graph())
        cpu, oc = cpu_alg1(adj_h, deg_h, base, info["nav"], q, kc, L)
        cpu["serial_scan"] = cpu_serial_scan(base, q)
        del adj_h, deg_h
        if base_form == "plain" or info["has_" + base_form] == 2:  # the oracle takes the same steps
            mq = len(oc["n_expand"])
            g_ne = cnt["n_expand"][:mq].cpu().numpy()
            g_nd = cnt["n_dist"][:mq].cpu().numpy()
            counts_check = {"queries": mq, "n_expand_equal": float((g_ne == oc["n_expand"]).mean()),
                            "n_dist_equal": float((g_nd == oc["n_dist"]).mean()),
                            "n_dist_gpu_over_oracle": float(g_nd.sum() / max(1, oc["n_dist"].sum()))}
            if mq == nq and "+stop" not in chosen_form:
                n_expand, n_dist = int(oc["n_expand"].sum()), int(oc["n_dist"].sum())
                bytes_launch = (n_dist * row_bytes + n_expand * R * 4 + nq * (d * 4 + kc * 8)
                                + (nq * L * d * 4 if lossy else 0))
                count_src = "oracle Alg. 1 on the same index and queries"

    peak, peak_kind = peaks()
    achieved = bytes_launch / (ms_step / 1e3) / 1e9
    src = kernel_source_hash()
    tr = NCU_TRAFFIC.get((src, args.workload, chosen_form, L))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": (tr * nq if tr else None),
                # the captured DRAM traffic over the same time: what HBM actually moved
                "dram_gbs": (tr * nq / (ms_step / 1e3) / 1e9 if tr else None),
                "peak_kind": peak_kind, "kernel": f"search_kernel ({chosen_form})",
                "algorithmic_bytes": bytes_launch, "kernel_src": src}
    # instruction issue: the search kernel is bound by it (ncu: ~73 % of active cycles
    # issue); warp instructions per launch over its time, against one instruction per
    # cycle per scheduler (4 per SM) at the maximum SM clock
    ins = NCU_INSTRUCTIONS.get((src, args.workload, chosen_form, L))
    issue_roofline = None
    if ins:
        props = torch.cuda.get_device_properties(0)
        mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
        ipeak = props.multi_processor_count * 4 * mhz * 1e6
        iach = ins * nq / (ms_step / 1e3)
        issue_roofline = {"bound": "issue", "achieved": iach, "peak": ipeak, "unit": "warp instructions/s",
                          "frac": iach / ipeak, "instructions_per_query": ins, "kernel_src": src,
                          "peak_from": "SMs x 4 schedulers x max SM clock"}
    # MRNG edge selection over the whole build: every examined candidate's id,
    # distance and FP32 row read once, the adjacency row, degree and candidate
    # count per node; over the prune launches' CUDA-event time
    prune_bytes = info["prune_examined"] * (4 * d + 8) + n * (4 * BUILD["R"] + 8)
    prune_roofline = {"bound": "hbm", "achieved": prune_bytes / (info["ms_prune"] / 1e3) / 1e9 if info["ms_prune"] else None,
                      "peak": peak, "unit": "GB/s", "peak_kind": peak_kind, "kernel": "prune_kernel",
                      "algorithmic_bytes": prune_bytes, "examined_per_node": info["prune_examined"] / n,
                      "ms": info["ms_prune"], "kernel_src": kernel_source_hash(PRUNE_SOURCES)}
    ptr = PRUNE_TRAFFIC.get((prune_roofline["kernel_src"], args.workload))
    prune_roofline["traffic"] = ptr * n if ptr else None
    if prune_roofline["achieved"] is not None:
        prune_roofline["frac"] = prune_roofline["achieved"] / peak

    # recall@10 of the chosen form and L on a second, held-out query batch
    # (L was picked on the timed batch)
    _, q_held = datagen.workload(args.workload, nq=nq, seed_query=datagen.SEED_QUERY + 7777 + 1000 * rank)
    qht = torch.from_numpy(q_held).cuda()
    gt_held, _ = ground_truth(capi, bt, qht, W)
    o_held = idx.search_ex(qht, kc, L, params=prm, counters=False)
    rec_held = capi.nsg_recall(o_held["ids"][:, :10].contiguous(), gt_held, 10).sum().item() / (10.0 * nq)
    del qht, gt_held, o_held


    if rank == 0:
        line = {
            "metric": METRIC, "value": job_qps(world, nq, ms_step), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"plain": "f32", "bf16": "bf16->f32", "fp8": "fp8e4m3->f32", "u8": "u8->i32"}[base_form],
            "data": "synthetic",
            "config": bench_config(W, world, base),
            "operating_point": {"form": chosen_form, "k": kc, "L": L, "recall10": rec_chosen,
                                "recall10_ties": rec_chosen_ties, "recall10_heldout": rec_held},
            "plain": {"value": job_qps(world, nq, ms_plain), "ms_per_step": ms_plain, "L": plain_L,
                      "recall10": rec_plain},
            "chosen_over_plain": ms_plain / ms_step,
            "roofline": roofline,
            "issue_roofline": issue_roofline,
            "prune_roofline": prune_roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": job_qps(world, nq, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": nq * d * 4, "d2h_bytes_per_step": nq * kc * 4,
                    "call": "nsg_search_host", "same_ids_as_device_call": e2e_same},
            # per step: the visiting order (distance, bucket, scan, scatter) and the search
            "gpu_launches": 5 * args.steps,
            "clocks": clocks,
            "build_seconds": build_s,
            "build_ms": {k: info[k] for k in ("ms_knn", "ms_centroid_nav", "ms_collect", "ms_prune",
                                               "ms_connect", "ms_total")},
            "index": {"avg_degree": info["avg_degree"], "max_degree": info["max_degree"],
                      "fixup_edges": info["n_fixup_edges"], "fixup_researched": info["n_fixup_searches"],
                      "nav": info["nav"], "bf16_exact": info["has_bf16"] == 2, "u8_exact": info["has_u8"] == 2,
                      "fp8_scale": info["fp8_scale"]},
            "per_query": {"n_expand": n_expand / nq, "n_dist": n_dist / nq, "source": count_src,
                          "gpu_counting_pass_vs_oracle": counts_check},
            "batched": batched,
            "partitioned": extras.get("partitioned"),
            "nndescent": extras.get("nndescent"),
            "nsg_naive": naive,
            "learned_stop": None if stop_loss is None else {
                "train_queries": nq, "trace_L": list(STOP_TRACE_LS), "iters": STOP_ITERS, "train_seconds": train_s,
                "loss_first": stop_loss[0].item(), "loss_last": stop_loss[-1].item(), "thresholds": STOP_THRESHOLDS},
            "precision_error_vs_fp64": prec_err,
            "at_recall10": at_recall,
            "sweep": sweeps,
        }
        if args.workload == "sift" and world == 1 and not (args.no_configs or args.compact):
            line["configs"] = config_runs(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
