"""Full-size (1,000,000 x 128, integer 0..255, 10,000 queries) checks in the
launch configuration the benchmark times.

The oracle cannot build a 1M-node graph in seconds, so it checks what it can
compute one unit at a time from its own inputs: sampled kNN rows (serial
scan), the centroid, the navigating node and sampled candidate lists /
pruned rows (its kNN rows computed lazily, only where its searches go).  The
finished graph and the search results are checked through properties that
hold at any size: out-degree <= R, every node reachable from the navigating
node, result keys sorted, exact distances, the closed final pool of Alg. 1,
and precision against the oracle's exact ground truth."""
import numpy as np
import pytest
import torch

import oracle
from checkers import reachable
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu

K, LB, R, CAP = 100, 40, 50, 500


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def sift():
    base, q = datagen.workload("sift")
    return base, q, T(base), T(q)


def test_fullsize_build_steps_sampled(nsg, sift):
    base, q, bt, qt = sift
    n = len(base)
    knn, kd2 = nsg.nsg_knn_init(bt, K)
    rows = np.array([0, 123457, n - 1], np.int64)
    rid, rd2 = oracle.knn_rows(base, K, rows=rows)
    assert np.array_equal(H(knn[rows]), rid)
    assert np.array_equal(H(kd2[rows]), rd2)

    c = nsg.nsg_centroid(bt)
    c_ref = oracle.centroid(base)
    assert np.array_equal(H(c), c_ref)

    start = oracle.start_node(0, n)
    nav = nsg.nsg_navigate(bt, knn, c, start, LB)
    lazy = oracle.LazyKnn(base, K)
    assert nav == lazy.navigate(c_ref, start, LB)

    for v in (7, 654321):
        ids, d2, cnt, st = nsg.nsg_collect(bt, knn, nav, LB, CAP, v0=v, nv=1)
        rids, rd2, rcnt = lazy.collect(nav, v, LB, CAP)
        assert int(H(cnt)[0]) == rcnt and int(H(st)[0]) == 0
        assert np.array_equal(H(ids)[0], rids)
        assert np.array_equal(H(d2)[0], rd2)
        adj, deg = nsg.nsg_prune(bt, ids, d2, cnt, R, v0=v)
        prow, pdeg = oracle.prune(base, rids[:rcnt], rd2[:rcnt], R)
        assert int(H(deg)[v]) == pdeg
        assert np.array_equal(H(adj)[v], prow)


@pytest.fixture(scope="module")
def index(nsg, sift):
    base, q, bt, qt = sift
    return nsg.nsg_build(bt, K, LB, R, CAP, seed=0)


def test_fullsize_graph_invariants(nsg, sift, index):
    base = sift[0]
    info = index.info()
    adj, deg = index.graph()
    adj, deg = H(adj), H(deg)
    assert info["n"] == len(base) and info["R"] == R
    assert (deg >= 1).all() and (deg <= R).all()
    assert reachable(adj, deg, info["nav"]).all()
    rng = np.random.default_rng(3)
    for v in rng.choice(len(base), 200, replace=False):
        row = adj[v][: deg[v]]
        assert (adj[v][deg[v]:] == -1).all()
        assert v not in row and len(set(row.tolist())) == len(row)


def test_fullsize_search_properties(nsg, sift, index):
    base, q, bt, qt = sift
    L = 100
    ids, d2 = index.search(qt, L, L)  # k = L: the whole final pool
    ids, d2 = H(ids), H(d2)
    adj, deg = index.graph()
    adj = H(adj)
    rng = np.random.default_rng(4)
    sample = rng.choice(len(q), 40, replace=False)
    for i in sample:
        keys = list(zip(d2[i].tolist(), ids[i].tolist()))
        assert keys == sorted(keys) and len(set(ids[i].tolist())) == L
        exact = ((base[ids[i]].astype(np.float64) - q[i]) ** 2).sum(1)
        assert np.array_equal(d2[i].astype(np.float64), exact)
        # closed pool: every out-neighbour of a pool entry is in the pool or beyond its tail
        pool = set(ids[i].tolist())
        tail = keys[-1]
        nb = np.unique(adj[ids[i]].ravel())
        nb = np.array([x for x in nb.tolist() if x >= 0 and x not in pool], np.int64)
        dn = ((base[nb].astype(np.float64) - q[i]) ** 2).sum(1)
        assert all((float(a), int(b)) > tail for a, b in zip(dn, nb))
    gt, _ = oracle.knn_query(base, q[sample], 10)
    assert oracle.recall(ids[sample][:, :10], gt, 10) >= 0.9


def test_fullsize_recall_sweep_monotone(nsg, sift, index):
    base, q, bt, qt = sift
    gt_ids, _ = nsg.nsg_knn_query(bt, qt[:2000], 10)
    sub = np.arange(0, 2000, 40)
    ref_gt, _ = oracle.knn_query(base, q[sub], 10)
    assert np.array_equal(H(gt_ids)[sub], ref_gt)
    prev = 0.0
    for L in (100, 200, 400):
        ids, _ = index.search(qt[:2000], 10, L)
        r = H(nsg.nsg_recall(ids, gt_ids, 10)).sum() / 20000.0
        assert r >= prev - 1e-3
        prev = r
    assert prev >= 0.95
