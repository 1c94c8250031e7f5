"""Oracle pins for Alg. 1 (Search-on-Graph)."""
import os

import numpy as np
import pytest

import oracle
from checkers import brute_knn, edges_of, read_golden, reachable
from paper_1707_00143_gb300 import datagen


def _golden_graph(golden_dir):
    recs = read_golden(os.path.join(golden_dir, "alg1_trace_small.txt"))
    pts, edges, cases, cur = {}, {}, [], None
    for tag, v in recs:
        if tag == "point":
            pts[int(v[0])] = [float(v[1]), float(v[2])]
        elif tag == "edges":
            edges[int(v[0])] = [int(x) for x in v[1:]]
        elif tag == "query":
            q = np.array([float(v[0]), float(v[1])], np.float32)
        elif tag == "start":
            start = int(v[0])
        elif tag == "case":
            cur = dict(l=int(v[1]), steps=[])
            cases.append(cur)
        elif tag == "step":
            cur["steps"].append([int(x) for x in v])
        elif tag in ("n_expand", "n_dist"):
            cur[tag] = int(v[0])
        elif tag == "result":
            cur["result"] = [int(x) for x in v]
    n = len(pts)
    base = np.array([pts[i] for i in range(n)], np.float32)
    adj = np.full((n, 3), -1, np.int32)
    for i, e in edges.items():
        adj[i, : len(e)] = e
    return base, adj, q, start, cases


def test_alg1_hand_trace(golden_dir):
    base, adj, q, start, cases = _golden_graph(golden_dir)
    for c in cases:
        tr = oracle.search_trace(adj, base, start, q, c["l"])
        assert tr.tolist() == [s + [-1] * (c["l"] - len(s)) for s in c["steps"]]
        ids, dist, ne, nd = oracle.search(adj, base, start, q[None], len(c["result"]), c["l"])
        assert ids[0].tolist() == c["result"]
        assert ne[0] == c["n_expand"] and nd[0] == c["n_dist"]


def _ring_plus_random(n, extra, seed):
    """Strongly connected graph: a ring plus random extra edges."""
    rng = np.random.default_rng(seed)
    adj = np.full((n, extra + 1), -1, np.int32)
    for i in range(n):
        nb = [(i + 1) % n] + [int(x) for x in rng.choice(n, size=extra, replace=False) if x != i]
        nb = list(dict.fromkeys(nb))
        adj[i, : len(nb)] = nb
    return adj


@pytest.mark.parametrize("hi", [256, 4])
def test_alg1_pool_at_least_n_is_serial_scan(hi):
    # With l >= n nothing is ever evicted, every reachable node is added and
    # checked, so the pool is the exact kNN of the reachable set (Sec. 4.1.2).
    n = 120
    base = datagen.uniform_int(n, 6, seed=21, hi=hi)
    q = datagen.uniform_int(15, 6, seed=22, hi=hi)
    adj = _ring_plus_random(n, 3, seed=23)
    ids, dist, ne, nd = oracle.search(adj, base, 7, q, 30, n)
    rid, rdist = brute_knn(base, q, 30)
    assert np.array_equal(ids, rid)
    assert np.array_equal(dist.astype(np.float64), rdist)
    assert (ne == n).all() and (nd == n).all()


def test_alg1_unreachable_part_is_never_returned():
    n = 60
    base = datagen.uniform_int(n, 4, seed=24)
    adj = _ring_plus_random(n, 2, seed=25)
    adj[adj >= 30] = -1  # nodes 30.. become unreachable from 0
    for i in range(30):
        row = [x for x in adj[i] if x >= 0] or [(i + 1) % 30]
        adj[i] = -1
        adj[i, : len(row)] = row
    deg = (adj >= 0).sum(1).astype(np.int32)
    mask = reachable(adj, deg, 0)
    assert mask[:30].all() and not mask[30:].any()
    q = datagen.uniform_int(5, 4, seed=26)
    ids, dist, ne, nd = oracle.search(adj, base, 0, q, 40, 100)
    assert (ids[:, :30] < 30).all() and (ids[:, :30] >= 0).all()
    assert (ids[:, 30:] == -1).all() and np.isinf(dist[:, 30:]).all()  # padded


def test_alg1_on_mrng_reaches_every_base_point_with_l1():
    # Thm 3 (MRNG is an MSNET) + Thm 1 (Alg. 1 finds a monotonic path without
    # backtracking): with pool size 1, the search from any node toward any
    # base point ends at that point.
    base = datagen.uniform_float(40, 3, seed=27)
    adj, deg = oracle.mrng_naive(base)
    for s in range(0, 40, 3):
        ids, dist, _, _ = oracle.search(adj, base, s, base, 1, 1, deg=deg)
        assert np.array_equal(ids[:, 0], np.arange(40))
        assert (dist[:, 0] == 0).all()


def test_alg1_final_pool_is_closed():
    # At termination every pool entry is checked, so each out-neighbour of a
    # pool entry is either in the pool or farther than the pool's last entry.
    base, q = datagen.workload("tiny", n=800, nq=10)
    knn, _ = oracle.knn_rows(base, 8)
    L = 20
    ids, dist, ne, nd = oracle.search(knn, base, 0, q, L, L)
    for i in range(len(q)):
        pool = set(ids[i].tolist())
        tail = (float(dist[i, -1]), int(ids[i, -1]))
        for u in ids[i]:
            for v in knn[u]:
                if int(v) in pool:
                    continue
                dv = float(((base[v].astype(np.float64) - q[i]) ** 2).sum())
                assert (dv, int(v)) > tail
