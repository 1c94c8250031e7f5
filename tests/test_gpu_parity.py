"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Integer-valued data (0..255) makes every float32 squared distance exact and
order-independent, so the CUDA path must reproduce the oracle bit for bit:
kNN graph, centroid, navigating node, candidate lists, pruned rows, fix-up
edges, the whole graph, and search ids / distances / step counts.  Sizes span
many tiles with ragged tails (n = 10,000 = 78 x 128 + 16; nq not a multiple
of the 32 queries per block or the warps per block)."""
import numpy as np
import pytest
import torch

import oracle
from checkers import reachable
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu

K, LB, R, CAP = 20, 40, 16, 200  # build parameters of the 10k x 32 workload


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    base, q = datagen.workload("tiny")
    ref = oracle.build(base, K, LB, R, CAP, seed=0)
    adj0, deg0 = oracle.select_all(ref["knn"], base, ref["nav"], LB, R, CAP)
    return dict(base=base, q=q, ref=ref, adj0=adj0, deg0=deg0)


def test_knn_init_bit_exact(nsg, tiny):
    base = tiny["base"]
    ids, d2 = nsg.nsg_knn_init(T(base), K)
    rid, rd2 = oracle.knn_rows(base, K)
    assert np.array_equal(H(ids), rid)
    assert np.array_equal(H(d2), rd2)


@pytest.mark.parametrize("k", [1, 10, 100])
def test_knn_query_bit_exact(nsg, tiny, k):
    base, q = tiny["base"], tiny["q"]
    q = q[:77]  # ragged: 2 blocks of 32 + 13
    ids, d2 = nsg.nsg_knn_query(T(base), T(q), k)
    rid, rd2 = oracle.knn_query(base, q, k)
    assert np.array_equal(H(ids), rid)
    assert np.array_equal(H(d2), rd2)


def test_centroid_bit_exact(nsg, tiny):
    c = nsg.nsg_centroid(T(tiny["base"]))
    assert np.array_equal(H(c), oracle.centroid(tiny["base"]))


def test_navigate_bit_exact(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    start = oracle.start_node(0, len(base))
    c = oracle.centroid(base)
    nav = nsg.nsg_navigate(T(base), T(ref["knn"]), T(c), start, LB)
    assert nav == ref["nav"] == oracle.navigate(ref["knn"], base, c, start, LB)


def test_collect_bit_exact(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    ids, d2, cnt, st = nsg.nsg_collect(T(base), T(ref["knn"]), ref["nav"], LB, CAP)
    ids, d2, cnt = H(ids), H(d2), H(cnt)
    assert (H(st) == 0).all()
    rng = np.random.default_rng(5)
    sample = np.concatenate([[0, ref["nav"], len(base) - 1], rng.choice(len(base), 400, replace=False)])
    for v in sample:
        rid, rd2, rc, _, _ = oracle.collect(ref["knn"], base, ref["nav"], int(v), LB, CAP)
        assert cnt[v] == rc
        assert np.array_equal(ids[v], rid), v
        assert np.array_equal(d2[v], rd2), v


def test_collect_then_prune_all_nodes_bit_exact(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    ids, d2, cnt, _ = nsg.nsg_collect(T(base), T(ref["knn"]), ref["nav"], LB, CAP)
    adj, deg = nsg.nsg_prune(T(base), ids, d2, cnt, R)
    assert np.array_equal(H(deg), tiny["deg0"])
    assert np.array_equal(H(adj), tiny["adj0"])


def test_prune_list_ends_at_negative_id(nsg, tiny):
    # counts of C with -1 padding after each list: the padding ends the list
    base, ref = tiny["base"], tiny["ref"]
    ids, d2, cnt, _ = nsg.nsg_collect(T(base), T(ref["knn"]), ref["nav"], LB, CAP)
    full = torch.full_like(cnt, CAP)
    adj, deg = nsg.nsg_prune(T(base), ids, d2, full, R)
    assert np.array_equal(H(deg), tiny["deg0"])
    assert np.array_equal(H(adj), tiny["adj0"])


def test_prune_chunked_offsets(nsg, tiny):
    # rows v0..v0+nv-1 only; other rows untouched
    base, ref = tiny["base"], tiny["ref"]
    v0, nv = 3001, 517
    ids, d2, cnt, _ = nsg.nsg_collect(T(base), T(ref["knn"]), ref["nav"], LB, CAP, v0=v0, nv=nv)
    adj, deg = nsg.nsg_prune(T(base), ids, d2, cnt, R, v0=v0)
    adj, deg = H(adj), H(deg)
    assert np.array_equal(adj[v0:v0 + nv], tiny["adj0"][v0:v0 + nv])
    assert (adj[:v0] == -1).all() and (adj[v0 + nv:] == -1).all() and (deg[:v0] == 0).all()


def test_connect_bit_exact(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    adj, deg = T(tiny["adj0"]), T(tiny["deg0"])
    added = nsg.nsg_connect(T(base), adj, deg, ref["nav"], LB)
    assert added == ref["n_added"]
    assert np.array_equal(H(adj), ref["adj"])
    assert np.array_equal(H(deg), ref["deg"])


def test_build_bit_exact(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    idx = nsg.nsg_build(T(base), K, LB, R, CAP, seed=0)
    info = idx.info()
    adj, deg = idx.graph()
    assert info["nav"] == ref["nav"]
    assert info["n_fixup_edges"] == ref["n_added"]
    assert np.array_equal(H(deg), ref["deg"])
    assert np.array_equal(H(adj), ref["adj"])
    assert reachable(H(adj), H(deg), info["nav"]).all()
    assert info["max_degree"] <= R


def test_build_prune_examined_count(nsg, tiny):
    # the edge selection examines a node's candidates in key order until R are
    # kept (then up to the R-th kept one) or the list ends; the oracle's
    # candidate lists and rows give that count per node
    base, ref = tiny["base"], tiny["ref"]
    want = 0
    for v in range(len(base)):
        cid, cd, cnt, _, _ = oracle.collect(ref["knn"], base, ref["nav"], v, LB, CAP)
        row, deg = oracle.prune(base, cid[:cnt], cd[:cnt], R)
        want += int(np.nonzero(cid[:cnt] == row[R - 1])[0][0]) + 1 if deg == R else cnt
    info = nsg.nsg_build(T(base), K, LB, R, CAP, seed=0).info()
    assert info["prune_examined"] == want


@pytest.mark.parametrize("k,L", [(10, 50), (1, 10), (16, 16), (100, 137), (10, 400), (10, 1024)])
def test_search_bit_exact(nsg, tiny, k, L):
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    params = nsg.SearchParams(0, 16384, nsg.PREC_F32, 0)  # visited set large enough never to forget
    out = idx.search_ex(T(q), k, L, params=params)
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, k, L, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)
    assert (H(out["status"]) == 0).all()


@pytest.mark.parametrize("hash_slots", [64, 16384])
def test_search_rows_listing_an_id_twice(nsg, tiny, hash_slots):
    # a caller's graph may list a neighbour twice in one row: Alg. 1 visits it
    # once (S is a set), so results equal the oracle's on the same rows; with
    # 64 slots the visited set is saturated and forgets, and the pool merge
    # drops the second copy when both lanes offer it
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    adj, deg = ref["adj"].copy(), ref["deg"].copy()
    rows = np.nonzero(deg < adj.shape[1])[0][::3]
    adj[rows, deg[rows]] = adj[rows, 0]
    deg[rows] += 1
    idx = nsg.nsg_index_from_graph(T(base), T(adj), ref["nav"], deg=T(deg))
    out = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, hash_slots, nsg.PREC_F32, 0))
    rid, rd2, rne, rnd = oracle.search(adj, base, ref["nav"], q, 10, 60, deg=deg)
    assert len(rows) > 100
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    if hash_slots == 16384:
        assert np.array_equal(H(out["n_dist"]), rnd)


@pytest.mark.parametrize("nq", [1, 31, 33, 100])
def test_search_default_params_and_ragged_batches(nsg, tiny, nq):
    # default (smaller, forgetful) visited set: ids / distances / steps unchanged
    base, q, ref = tiny["base"], tiny["q"][:nq], tiny["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"])
    ids, d2 = idx.search(T(q), 10, 50)
    out = idx.search_ex(T(q), 10, 50)
    rid, rd2, rne, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 50)
    assert np.array_equal(H(ids), rid) and np.array_equal(H(d2), rd2)
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["n_expand"]), rne)


def test_search_tiny_hash_forgets_but_results_hold(nsg, tiny):
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"])
    out = idx.search_ex(T(q), 10, 200, params=nsg.SearchParams(0, 64, nsg.PREC_F32, 0))
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, 10, 200)
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert (H(out["n_dist"]) >= rnd).all() and (H(out["n_dist"]) > rnd).any()


def test_recall_kernel(nsg, tiny):
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    gt, _ = oracle.knn_query(base, q, 10)
    ids, _, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 30)
    hits = nsg.nsg_recall(T(ids), T(gt), 10)
    assert H(hits).sum() / (10.0 * len(q)) == oracle.recall(ids, gt, 10)


def test_step_cap_reports_status(nsg, tiny):
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"])
    out = idx.search_ex(T(q), 10, 50, params=nsg.SearchParams(2, 0, nsg.PREC_F32, 0))
    assert (H(out["status"]) == nsg.NSG_ESTEPCAP).all()
    assert (H(out["n_expand"]) == 2).all()


def test_save_load_roundtrip(nsg, tiny, tmp_path):
    base, q, ref = tiny["base"], tiny["q"], tiny["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"])
    p = str(tmp_path / "tiny.nsg")
    idx.save(p)
    idx2 = nsg.nsg_load(p)
    a, b = idx.search(T(q), 10, 50), idx2.search(T(q), 10, 50)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert idx2.info()["nav"] == ref["nav"]


def test_out_of_range_ids_rejected(nsg, tiny):
    base, ref = tiny["base"], tiny["ref"]
    bad = ref["adj"].copy()
    bad[17, 0] = len(base)
    with pytest.raises(nsg.NsgError) as e:
        nsg.nsg_index_from_graph(T(base), T(bad), ref["nav"])
    assert e.value.status == nsg.NSG_EINVAL


@pytest.mark.parametrize("hi,d,dups", [(4, 8, 300), (256, 6, 50)])
def test_ties_duplicates_and_unpadded_d(nsg, hi, d, dups):
    # few distinct values: massive exact distance ties (order decided by id);
    # duplicated rows: zero distances between distinct ids; d = 6: row padding
    base = datagen.duplicate_rows(datagen.uniform_int(3000, d, seed=51, hi=hi), dups, seed=52)
    q = datagen.uniform_int(45, d, seed=53, hi=hi)
    ref = oracle.build(base, 12, 30, 10, 60, seed=7)
    kid, kd2 = nsg.nsg_knn_init(T(base), 12)
    rid, rd2 = oracle.knn_rows(base, 12)
    assert np.array_equal(H(kid), rid) and np.array_equal(H(kd2), rd2)
    idx = nsg.nsg_build(T(base), 12, 30, 10, 60, seed=7)
    adj, deg = idx.graph()
    assert idx.info()["nav"] == ref["nav"]
    assert np.array_equal(H(adj), ref["adj"]) and np.array_equal(H(deg), ref["deg"])
    ids, d2 = idx.search(T(q), 10, 40)
    sid, sd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 40)
    assert np.array_equal(H(ids), sid) and np.array_equal(H(d2), sd2)


def test_small_graph_pads_results(nsg):
    # fewer reachable nodes than k: ids -1 and distances +inf past the pool
    base = datagen.uniform_int(6, 4, seed=54)
    adj = np.array([[1, -1], [0, -1], [-1, -1], [-1, -1], [-1, -1], [-1, -1]], np.int32)
    idx = nsg.nsg_index_from_graph(T(base), T(adj), 0)
    ids, d2 = idx.search(T(base[:3]), 4, 4)
    ids, d2 = H(ids), H(d2)
    assert (ids[:, 2:] == -1).all() and np.isinf(d2[:, 2:]).all()
    assert set(ids[0, :2]) == {0, 1}


@pytest.mark.parametrize("d,hi", [(600, 64), (1500, 32)])
def test_wide_rows_search_bit_exact(nsg, d, hi):
    # rows wider than 512 values take the wide search kernels (8 and 16 float4
    # slices per lane); integer data small enough that every squared distance
    # stays below 2^24 keeps FP32 exact, so the results are the oracle's
    base = datagen.uniform_int(2500, d, seed=d, hi=hi)
    q = datagen.uniform_int(70, d, seed=d + 1, hi=hi)
    ref = oracle.build(base, 12, 30, 12, 100, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    out = idx.search_ex(T(q), 10, 48, params=nsg.SearchParams(0, 16384, nsg.PREC_F32, 0))
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, 10, 48, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)
    # the low-precision wide kernels: BF16 and 8-bit copies hold these values
    # exactly and their sums stay below 2^24, so the traversal keys are the
    # FP32 ones and, with the FP32 re-rank, so are the results
    for prec in (nsg.PREC_BF16, nsg.PREC_U8):
        idx.prepare(prec)
        lp = idx.search_ex(T(q), 10, 48, params=nsg.SearchParams(0, 16384, prec, 0, 1))
        assert np.array_equal(H(lp["ids"]), rid) and np.array_equal(H(lp["d2"]), rd2)
        assert np.array_equal(H(lp["n_expand"]), rne)
    # and the GPU build of the same rows equals the oracle's graph
    g = nsg.nsg_build(T(base), 12, 30, 12, 100, seed=0)
    adj, deg = g.graph()
    assert g.info()["nav"] == ref["nav"]
    assert np.array_equal(H(deg), ref["deg"]) and np.array_equal(H(adj), ref["adj"])


def test_float_rows_search_within_tolerance(nsg):
    # float data: distances agree to 1e-5 relative; ids may differ only at
    # near-ties, so recall against the oracle's ids stays within 0.001
    base, q = datagen.workload("gist", n=3000, nq=60)
    ref = oracle.build(base, 16, 40, 24, 150, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    out = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 16384, nsg.PREC_F32, 0))
    rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 60, deg=ref["deg"])
    ids, d2 = H(out["ids"]), H(out["d2"])
    assert np.allclose(d2, rd2, rtol=1e-5, atol=0)
    assert oracle.recall(ids, rid, 10) >= 1.0 - 0.001
