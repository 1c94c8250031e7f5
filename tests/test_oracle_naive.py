"""Oracle pins for the NSG-Naive baseline (Section 4.1.2): MRNG edge selection
over the kNN graph's edges, searched by Alg. 1 with random initialisation.

Pinned against brute force and the definitions, not against the oracle's own
routines: the first kept edge of every node is its exact nearest neighbour,
kept edges lie in the node's exact K-nearest list in key order, no kept edge
is occluded by an earlier kept one, every rejected candidate before the last
keep has an occluder among the earlier keeps, and with a pool at least n on
a graph where every node reaches every other the search is the serial scan."""
import numpy as np

import oracle
from checkers import brute_knn, sqdist_matrix
from paper_1707_00143_gb300 import datagen


def test_naive_edges_follow_the_definition():
    base = datagen.uniform_int(400, 6, seed=91, hi=12)  # many exact ties
    K, R = 24, 8
    adj, deg = oracle.build_naive(base, K, R)
    D = sqdist_matrix(base, base)
    rid, _ = brute_knn(base, base, K, exclude_self=True)
    assert (deg >= 1).all() and (deg <= R).all()
    for v in range(len(base)):
        row = adj[v, :deg[v]].tolist()
        assert (adj[v, deg[v]:] == -1).all()
        cand = rid[v].tolist()
        assert row[0] == cand[0]  # nearest neighbour kept first
        pos = [cand.index(w) for w in row]
        assert pos == sorted(pos)  # kept edges in key order, all from the K nearest
        for a in range(len(row)):  # no kept edge occluded by an earlier kept one
            for b in range(a):
                assert not D[row[a], row[b]] < D[v, row[a]]
        for t in range(pos[-1] + 1):  # rejected candidates have an earlier occluder
            q = cand[t]
            if q in row:
                continue
            earlier = [w for w in row if cand.index(w) < t]
            assert any(D[q, r] < D[v, q] for r in earlier)


def test_random_init_with_full_pool_is_serial_scan():
    base = datagen.uniform_int(300, 8, seed=92)
    q = datagen.uniform_int(25, 8, seed=93)
    n = len(base)
    adj = np.array([[w for w in range(n) if w != v] for v in range(n)], np.int32)  # complete graph
    ids, d2, ne, nd = oracle.search_random(adj, base, q, 10, n, 16, seed=7)
    rid, rd2 = brute_knn(base, q, 10)
    assert np.array_equal(ids, rid) and np.array_equal(d2, rd2)
    assert (nd == n).all()  # every node's distance computed exactly once


def test_random_init_draws_match_the_stated_generator():
    # with one draw the pool starts at splitmix64(seed + q * golden) mod n:
    # the same search as Alg. 1 from that start node
    base, q = datagen.workload("tiny", n=2000, nq=12)
    ref = oracle.build(base, 16, 30, 12, 100, seed=0)
    seed, golden = 11, 0x9E3779B97F4A7C15
    a = oracle.search_random(ref["adj"], base, q, 10, 40, 1, seed, deg=ref["deg"])
    for i in range(len(q)):
        start = oracle.splitmix64((seed + i * golden) % (1 << 64)) % len(base)
        b = oracle.search(ref["adj"], base, start, q[i:i + 1], 10, 40, deg=ref["deg"])
        assert np.array_equal(a[0][i], b[0][0]) and a[2][i] == b[2][0] and a[3][i] == b[3][0]
