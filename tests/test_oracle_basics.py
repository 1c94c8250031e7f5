"""Oracle pins: distance, start-node generator, centroid, serial-scan kNN, precision."""
import os

import numpy as np
import pytest

import oracle
from checkers import brute_knn, precision, read_golden
from paper_1707_00143_gb300 import datagen


def test_dist2_closed_forms():
    # 3-4-5 triangle and a 1-D case, by hand
    assert oracle.dist2([0, 0], [3, 4]) == 25.0
    assert oracle.dist2([7], [2]) == 25.0
    assert oracle.dist2([1, 2, 3], [1, 2, 3]) == 0.0


def test_dist2_exact_on_integer_data():
    # integer coordinates 0..255, d <= 258: every partial sum is an integer < 2^24,
    # so the float sum equals the exact (float64) sum in any order.
    x = datagen.uniform_int(64, 128, seed=5)
    for i in range(0, 64, 2):
        exact = float(((x[i].astype(np.float64) - x[i + 1]) ** 2).sum())
        assert oracle.dist2(x[i], x[i + 1]) == exact
        assert oracle.dist2(x[i + 1], x[i]) == exact  # symmetric


def test_splitmix64_published_vectors(golden_dir):
    for tag, vals in read_golden(os.path.join(golden_dir, "splitmix64.txt")):
        assert oracle.splitmix64(int(tag, 16)) == int(vals[0], 16)


def test_centroid_exact_on_integers():
    x = datagen.uniform_int(1000, 16, seed=7)
    c = oracle.centroid(x)
    # integer column sums are exact in double; the division is correctly rounded
    ref = x.astype(np.int64).sum(0).astype(np.float64) / 1000.0
    assert np.array_equal(c, ref)


def test_centroid_float_within_rounding():
    import math

    x = datagen.uniform_float(500, 8, seed=8)
    c = oracle.centroid(x)
    ref = np.array([math.fsum(map(float, x[:, j])) / 500 for j in range(8)])
    assert np.allclose(c, ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("hi", [256, 3])  # hi=3: massive distance ties
def test_knn_rows_vs_lexsort(hi):
    x = datagen.uniform_int(300, 8, seed=11, hi=hi)
    ids, dist = oracle.knn_rows(x, 10, nthreads=3)
    rid, rdist = brute_knn(x, x, 10, exclude_self=True)
    assert np.array_equal(ids, rid)
    assert np.array_equal(dist.astype(np.float64), rdist)


def test_knn_rows_duplicates_stay_neighbours():
    x = datagen.duplicate_rows(datagen.uniform_int(200, 4, seed=12), 30, seed=13)
    ids, dist = oracle.knn_rows(x, 5)
    rid, _ = brute_knn(x, x, 5, exclude_self=True)
    assert np.array_equal(ids, rid)
    assert all(ids[i, 0] != i for i in range(200))  # self excluded by id, not by distance
    dup = [i for i in range(200) if dist[i, 0] == 0.0]
    assert dup  # duplicated points are each other's nearest neighbour at distance 0


def test_knn_threads_do_not_change_result():
    x = datagen.uniform_int(400, 8, seed=14, hi=5)
    a, _ = oracle.knn_rows(x, 7, nthreads=1)
    b, _ = oracle.knn_rows(x, 7, nthreads=5)
    c, _ = oracle.knn_rows(x, 7, rows=np.arange(400), nthreads=7)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_knn_query_vs_lexsort():
    b = datagen.uniform_int(500, 16, seed=15, hi=16)
    q = datagen.uniform_int(40, 16, seed=16, hi=16)
    ids, dist = oracle.knn_query(b, q, 20)
    rid, rdist = brute_knn(b, q, 20)
    assert np.array_equal(ids, rid)
    assert np.array_equal(dist.astype(np.float64), rdist)


def test_knn_k_larger_than_rows_pads():
    x = datagen.uniform_int(5, 4, seed=17)
    ids, dist = oracle.knn_rows(x, 6)
    assert (ids[:, 4:] == -1).all() and np.isinf(dist[:, 4:]).all()


def test_recall_matches_definition():
    rng = np.random.default_rng(0)
    gt = np.stack([rng.permutation(50)[:10] for _ in range(20)]).astype(np.int32)
    ids = gt.copy()
    ids[:, 5:] = rng.integers(50, 100, size=(20, 5))
    assert oracle.recall(ids, gt, 10) == 0.5
    assert oracle.recall(ids, gt, 10) == precision(ids, gt, 10)
    # hand case: 2 of 3 ids found
    assert oracle.recall(np.array([[1, 2, 9]]), np.array([[2, 1, 3]]), 3) == pytest.approx(2 / 3)
