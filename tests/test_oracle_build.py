"""Oracle pins for Alg. 2 (NSGbuild): centroid/navigating node, search-and-collect,
connectivity pass, and whole-build invariants."""
import numpy as np
import pytest

import oracle
from checkers import brute_knn, occlusion_violations, reachable, sqdist_matrix
from paper_1707_00143_gb300 import datagen


def _connected_graph(n, K, seed):
    rng = np.random.default_rng(seed)
    g = np.empty((n, K), np.int32)
    for i in range(n):
        nxt = (i + 1) % n
        others = rng.permutation(np.setdiff1d(np.arange(n), [i, nxt]))[: K - 1]
        g[i] = np.concatenate([[nxt], others])
    return g


def test_collect_with_pool_n_is_exact_neighbourhood():
    # l >= n: the search visits every node reachable from nav (all of them),
    # so E = all nodes but v and its first C entries are v's exact C nearest.
    n = 150
    base = datagen.uniform_int(n, 5, seed=41, hi=8)
    g = _connected_graph(n, 4, seed=42)
    Cap = 40
    for v in (0, 17, 149):
        ids, dist, cnt, ne, nd = oracle.collect(g, base, 3, v, n, Cap)
        rid, rdist = brute_knn(base, base, Cap, exclude_self=True)
        assert cnt == Cap and ne == n and nd == n
        assert ids.tolist() == rid[v].tolist()
        assert np.array_equal(dist.astype(np.float64), rdist[v])


def test_collect_contains_knn_row_and_excludes_v():
    base, _ = datagen.workload("tiny", n=1500, nq=1)
    knn, _ = oracle.knn_rows(base, 10)
    for v in (0, 5, 999):
        ids, dist, cnt, ne, nd = oracle.collect(knn, base, 0, v, 20, 1000)
        got = ids[:cnt]
        assert v not in got.tolist()
        assert len(set(got.tolist())) == cnt  # unique
        assert set(knn[v].tolist()) <= set(got.tolist())  # Alg. 2: v's kNN neighbours join the candidates
        keys = list(zip(dist[:cnt].tolist(), got.tolist()))
        assert keys == sorted(keys)  # Alg. 2: candidates sorted by key
        # every distance is the exact squared distance to x_v (integer data)
        exact = ((base[got].astype(np.float64) - base[v]) ** 2).sum(1)
        assert np.array_equal(dist[:cnt].astype(np.float64), exact)
        # the cap keeps the C smallest of the same set
        ids2, dist2, cnt2, _, _ = oracle.collect(knn, base, 0, v, 20, 30)
        assert cnt2 == min(30, cnt) and ids2[:cnt2].tolist() == got[:cnt2].tolist()


def test_navigate_with_pool_n_is_medoid_of_centroid():
    base = datagen.uniform_float(200, 6, seed=43)
    g = _connected_graph(200, 5, seed=44)
    c = oracle.centroid(base)
    nav = oracle.navigate(g, base, c, r=17, L=200)
    ref = np.argmin(((base.astype(np.float64) - c) ** 2).sum(1))
    assert nav == ref


def test_connect_on_empty_graph_attaches_to_nearest_reached():
    # No edges and an uncapped degree: every pass of the loop attaches the
    # smallest unreached id u to the nearest (by key) node reached so far,
    # because with l >= n Alg. 1 returns every reached node sorted by distance.
    n = 40
    base = datagen.uniform_int(n, 3, seed=45, hi=6)
    adj = np.full((n, n - 1), -1, np.int32)
    deg = np.zeros(n, np.int32)
    nav = 11
    adj2, deg2, added = oracle.connect(adj, deg, base, nav, L=n)
    D = sqdist_matrix(base, base)
    reached = [nav]
    expect = []
    for u in range(n):
        if u == nav:
            continue
        s = min(reached, key=lambda r: (D[r, u], r))
        expect.append((s, u))
        reached.append(u)
    assert [tuple(x) for x in added.tolist()] == expect


def test_connect_degree_fallback_and_error():
    base = np.array([[0, 0], [5, 0], [10, 0], [0, 1]], np.float32)
    adj = np.array([[1], [2], [-1], [-1]], np.int32)
    deg = np.array([1, 1, 0, 0], np.int32)
    # l = 1: the pool ends as [0] whose degree is full -> smallest reached id with room (2)
    _, deg2, added = oracle.connect(adj, deg, base, 0, L=1)
    assert added.tolist() == [[2, 3]] and deg2.tolist() == [1, 1, 1, 0]
    # all reached nodes full -> error
    cyc = np.array([[1], [2], [0], [-1]], np.int32)
    with pytest.raises(RuntimeError):
        oracle.connect(cyc, np.array([1, 1, 1, 0], np.int32), base, 0, L=4)


@pytest.fixture(scope="module")
def tiny_build():
    base, q = datagen.workload("tiny", n=2500, nq=50)
    K, L, R, Cap = 20, 40, 16, 200
    out = oracle.build(base, K, L, R, Cap, seed=0)
    return base, q, (K, L, R, Cap), out


def test_build_invariants(tiny_build):
    base, q, (K, L, R, Cap), out = tiny_build
    adj, deg, nav = out["adj"], out["deg"], out["nav"]
    assert (deg <= R).all() and (deg >= 1).all()
    assert reachable(adj, deg, nav).all()  # SCC = 1 as defined for fixed-start graphs
    for v in range(len(base)):  # no self loops, no repeated edges
        row = adj[v][: deg[v]].tolist()
        assert v not in row and len(set(row)) == len(row)
        assert (adj[v][deg[v]:] == -1).all()


def test_build_steps_compose(tiny_build):
    base, q, (K, L, R, Cap), out = tiny_build
    knn, _ = oracle.knn_rows(base, K)
    assert np.array_equal(knn, out["knn"])
    c = oracle.centroid(base)
    nav = oracle.navigate(knn, base, c, oracle.start_node(0, len(base)), L)
    assert nav == out["nav"]
    adj0, deg0 = oracle.select_all(knn, base, nav, L, R, Cap)
    # connectivity only appends edges: every selected row is a prefix of the final row
    for v in range(len(base)):
        assert out["adj"][v][: deg0[v]].tolist() == adj0[v][: deg0[v]].tolist()
    assert int((out["deg"] - deg0).sum()) == out["n_added"]
    assert occlusion_violations(base, adj0, deg0) == []
    # NNG subset of NSG with an exact kNN graph: the first kept edge is the exact NN
    assert (adj0[:, 0] == knn[:, 0]).all()


def test_build_thread_count_invariant():
    base, _ = datagen.workload("tiny", n=700, nq=1)
    a = oracle.build(base, 12, 30, 10, 100, seed=3, nthreads=1)
    b = oracle.build(base, 12, 30, 10, 100, seed=3, nthreads=6)
    assert np.array_equal(a["adj"], b["adj"]) and a["nav"] == b["nav"]


def test_search_on_build_beats_random_start(tiny_build):
    # sanity of the whole pipeline at tiny scale (not a paper number)
    base, q, (K, L, R, Cap), out = tiny_build
    gt, _ = oracle.knn_query(base, q, 10)
    ids, dist, ne, nd = oracle.search(out["adj"], base, out["nav"], q, 10, 60, deg=out["deg"])
    assert oracle.recall(ids, gt, 10) > 0.8
