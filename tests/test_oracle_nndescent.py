"""Pins of the oracle's nn-descent (the approximate kNN graph of Sec. 3.5 (ii),
Dong, Charikar and Li's method made deterministic), against what the method
and the mathematics fix:

* no iteration: every list is the seeded random draw (first K distinct ids
  != v of splitmix64(seed + v * 0x9e3779b97f4a7c15 + t) mod n), sorted by key;
* every list, after any number of iterations: K distinct ids, no self, sorted
  by (d2, id), each d2 the exact squared distance (integer data);
* each iteration keeps the K smallest keys of a superset of the list, so no
  list position ever gets a larger key;
* K = n - 1: the initial lists already hold every other node, so the result
  is the exact kNN graph from the start;
* the local join is the push form of the published method: one iteration
  recomputed here from its definition (samples, reverse samples, every pair
  of a join set offered to each other) gives the same lists;
* convergence: on clustered data the graph reaches the exact kNN graph up to
  a few entries, and a planted mistake (reverse samples dropped) converges
  measurably worse."""
import numpy as np
import pytest

import oracle
from paper_1707_00143_gb300 import datagen

GOLD = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _exact_d2(base, i, j):
    t = base[i].astype(np.int64) - base[j].astype(np.int64)
    return float((t * t).sum())


def _draw(n, K, seed, v):
    got, t = [], 0
    while len(got) < K:
        x = oracle.splitmix64((seed + v * GOLD + t) & M64) % n
        t += 1
        if x != v and x not in got:
            got.append(x)
    return got


@pytest.fixture(scope="module")
def small():
    base, _ = datagen.workload("tiny", n=600, nq=1)
    return base


def test_no_iteration_is_the_seeded_draw(small):
    base = small
    K, seed = 8, 5
    ids, d2, it, _ = oracle.nndescent(base, K, iters=0, seed=seed)
    assert it == 0
    for v in range(0, len(base), 37):
        want = sorted((_exact_d2(base, v, x), x) for x in _draw(len(base), K, seed, v))
        assert [x for _, x in want] == ids[v].tolist()
        assert [dd for dd, _ in want] == d2[v].astype(np.float64).tolist()


@pytest.mark.parametrize("iters", [1, 3, 8])
def test_lists_are_valid_knn_rows(small, iters):
    base = small
    K = 10
    ids, d2, _, _ = oracle.nndescent(base, K, S=6, Sr=6, iters=iters, seed=2)
    for v in range(len(base)):
        row = ids[v]
        assert len(set(row.tolist())) == K and v not in row
        keys = list(zip(d2[v].astype(np.float64), row))
        assert keys == sorted(keys)
        assert all(d2[v][i] == _exact_d2(base, v, row[i]) for i in range(K))


def test_no_list_position_ever_worsens(small):
    base = small
    prev = None
    for t in range(0, 6):
        _, d2, _, _ = oracle.nndescent(base, 12, S=4, Sr=4, iters=t, delta=-1.0, seed=3)
        if prev is not None:
            assert (d2 <= prev).all()
            assert (d2 < prev).any() or t > 3
        prev = d2


def test_all_other_nodes_known_from_the_start():
    base = datagen.uniform_int(40, 6, seed=11, hi=32)
    K = len(base) - 1
    ids, d2, _, _ = oracle.nndescent(base, K, S=4, Sr=4, iters=2, seed=1)
    gid, gd = oracle.knn_rows(base, K)
    assert np.array_equal(ids, gid) and np.array_equal(d2, gd)


def _one_iteration_push(base, ids, d2, isnew, S, Sr):
    """One iteration from the method's definition: samples, reverse samples,
    local join offering every pair of a join set to each other, lists cut to
    the K smallest keys of themselves and their offers."""
    n, K = ids.shape
    newS = [[ids[v][i] for i in range(K) if isnew[v][i]][:S] for v in range(n)]
    oldS = [[ids[v][i] for i in range(K) if not isnew[v][i]][:S] for v in range(n)]
    key = {(v, ids[v][i]): float(d2[v][i]) for v in range(n) for i in range(K)}
    rnew = [[] for _ in range(n)]
    rold = [[] for _ in range(n)]
    for v in range(n):
        for u in newS[v]:
            rnew[u].append((key[(v, u)], v))
        for u in oldS[v]:
            rold[u].append((key[(v, u)], v))
    offers = [dict() for _ in range(n)]
    for v in range(n):
        NEW = list(dict.fromkeys(newS[v] + [x for _, x in sorted(rnew[v])[:Sr]]))
        OLD = [x for x in dict.fromkeys(oldS[v] + [x for _, x in sorted(rold[v])[:Sr]]) if x not in NEW]
        for p in NEW:
            for q in NEW + OLD:
                if q != p:
                    dd = _exact_d2(base, p, q)
                    offers[p][q] = dd
                    offers[q][p] = dd
    out_ids = np.empty_like(ids)
    for p in range(n):
        cand = {int(ids[p][i]): float(d2[p][i]) for i in range(K)}
        for q, dd in offers[p].items():
            cand.setdefault(q, dd)
        out_ids[p] = [q for _, q in sorted((dd, q) for q, dd in cand.items())[:K]]
    return out_ids


def test_one_iteration_equals_the_push_form_of_the_local_join():
    base = datagen.uniform_int(120, 5, seed=12, hi=64)
    K, S, Sr = 6, 3, 2
    ids0, d20, _, _ = oracle.nndescent(base, K, S=S, Sr=Sr, iters=0, seed=4)
    ids1, _, _, _ = oracle.nndescent(base, K, S=S, Sr=Sr, iters=1, delta=-1.0, seed=4)
    want = _one_iteration_push(base, ids0, d20, np.ones_like(ids0, dtype=bool), S, Sr)
    assert np.array_equal(ids1, want)


def test_converges_near_the_exact_graph():
    base, _ = datagen.workload("tiny", n=3000, nq=1)
    K = 16
    gid, _ = oracle.knn_rows(base, K)
    ids, _, it, upd = oracle.nndescent(base, K, S=8, Sr=16, iters=15, delta=0.0, seed=9)
    recall = np.mean([len(set(ids[v]) & set(gid[v])) / K for v in range(len(base))])
    assert recall >= 0.97, recall
    # without reverse samples the join sees far fewer pairs per iteration
    ids_nr, _, _, _ = oracle.nndescent(base, K, S=8, Sr=0, iters=4, delta=0.0, seed=9)
    ids_r, _, _, _ = oracle.nndescent(base, K, S=8, Sr=16, iters=4, delta=0.0, seed=9)
    r_nr = np.mean([len(set(ids_nr[v]) & set(gid[v])) / K for v in range(len(base))])
    r_r = np.mean([len(set(ids_r[v]) & set(gid[v])) / K for v in range(len(base))])
    assert r_r > r_nr + 0.02, (r_r, r_nr)
