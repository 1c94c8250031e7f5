"""Batched uneven queries: per-query (k, L) in one persistent launch with a
device work queue; plans autotune the launch shape and replay a CUDA graph.

The plain form is the reference: every query's result must equal the fixed
(k, L) search of that query alone (ids and distances bit for bit on integer
data, whatever launch shape or visited-hash size the autotuner picks)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def setup(nsg):
    base, q = datagen.workload("tiny", n=8000, nq=300)
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    k, L = datagen.uneven_k_L(len(q), seed=91, ks=(1, 10, 50), l_lo=20, l_hi=200)
    return base, q, ref, idx, k, L


def _expect(idx, nsg, q, k, L, kmax, params=None):
    ids = np.full((len(q), kmax), -1, np.int32)
    d2 = np.full((len(q), kmax), np.inf, np.float32)
    for kk, LL in sorted(set(zip(k.tolist(), L.tolist()))):
        sel = np.nonzero((k == kk) & (L == LL))[0]
        out = idx.search_ex(T(q[sel]), kk, LL, params=params, counters=False)
        ids[sel, :kk] = H(out["ids"])
        d2[sel, :kk] = H(out["d2"])
    return ids, d2


def test_batched_equals_per_query_search(nsg, setup):
    base, q, ref, idx, k, L = setup
    out = idx.search_batched(T(q), T(k), T(L))
    ids, d2 = _expect(idx, nsg, q, k, L, int(k.max()))
    assert np.array_equal(H(out["ids"]), ids)
    assert np.array_equal(H(out["d2"]), d2)
    assert (H(out["status"]) == 0).all()
    # and equal to the oracle for a sample of queries
    for i in range(0, len(q), 37):
        rid, _, _, _ = oracle.search(ref["adj"], base, ref["nav"], q[i:i + 1], int(k[i]), int(L[i]))
        assert H(out["ids"])[i, :k[i]].tolist() == rid[0].tolist()


def test_plan_autotunes_and_replays(nsg, setup):
    base, q, ref, idx, k, L = setup
    qt, kt, Lt = T(q), T(k), T(L)
    plan = idx.plan(qt, kt, Lt, autotune=True)
    info = plan.info()
    # 24 shapes in shared memory and 24 with global-memory pools
    assert info["n_tried"] == 48 and info["warps_per_cta"] in (2, 4, 8) and info["warps_per_query"] in (1, 2, 4)
    assert info["pool"] in (1, 2)
    assert info["hash_slots"] in (512, 1024, 2048) and 0 < info["best_ms"] <= info["worst_ms"]
    ids, d2 = _expect(idx, nsg, q, k, L, int(k.max()))
    for _ in range(2):
        plan.ids.fill_(7)
        got_ids, got_d2 = plan.run()
        torch.cuda.synchronize()
        assert np.array_equal(H(got_ids), ids) and np.array_equal(H(got_d2), d2)
    # bound buffers: new query contents, same graph
    q2 = datagen.workload("tiny", n=10, nq=300, seed_query=92)[1]
    qt.copy_(T(q2))
    got_ids, _ = plan.run()
    ids2, _ = _expect(idx, nsg, q2, k, L, int(k.max()))
    assert np.array_equal(H(got_ids), ids2)


def test_batched_precision_and_stop_params(nsg, setup):
    base, q, ref, idx, k, L = setup
    idx.prepare(nsg.PREC_BF16)
    prm = nsg.SearchParams(0, 0, nsg.PREC_BF16)
    out = idx.search_batched(T(q), T(k), T(L), params=prm)
    ids, d2 = _expect(idx, nsg, q, k, L, int(k.max()), params=prm)
    assert np.array_equal(H(out["ids"]), ids) and np.array_equal(H(out["d2"]), d2)


def test_batched_rejects_bad_shapes(nsg, setup):
    base, q, ref, idx, k, L = setup
    with pytest.raises(nsg.NsgError):
        idx.search_batched(T(q), T(k), T(L), kmax=10, Lmax=5)  # Lmax < kmax
