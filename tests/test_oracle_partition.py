"""Pins of the oracle's partition-and-merge search (Sections 4.2, 4.3: the base
split at random into subsets, one NSG per subset, every query searched on
each, the results merged by key), against brute force, a hand-worked case
and the one-subset identity."""
import numpy as np
import pytest

import oracle
from paper_1707_00143_gb300 import datagen


def brute(base, q, k):
    d2 = ((q[:, None, :].astype(np.float64) - base[None, :, :].astype(np.float64)) ** 2).sum(-1)
    ids = np.stack([np.lexsort((np.arange(len(base)), row))[:k] for row in d2])
    return ids.astype(np.int32), np.take_along_axis(d2, ids, 1)


def test_even_partition_sizes_and_determinism():
    part = datagen.even_partition(1001, 4, seed=3)
    sizes = np.bincount(part, minlength=4)
    assert sizes.sum() == 1001 and sizes.max() - sizes.min() <= 1
    assert np.array_equal(part, datagen.even_partition(1001, 4, seed=3))
    assert not np.array_equal(part, datagen.even_partition(1001, 4, seed=4))


def test_hand_worked_two_subsets():
    # 1-D points, subsets {0, 2, 4} at x = 0, 4, 8 and {1, 3, 5} at x = 1, 5, 9;
    # query x = 4.25: distances 0.0625 (id 2), 0.5625 (id 3), 10.5625 (id 1)
    base = np.array([[0], [1], [4], [5], [8], [9]], np.float32)
    part = np.array([0, 1, 0, 1, 0, 1])
    q = np.array([[4.25]], np.float32)
    ids, d2 = oracle.partition_search(base, q, part, K=2, L_build=3, R=2, Cap=3, k=3, L=3)
    assert ids.tolist() == [[2, 3, 1]]
    assert d2.tolist() == [[0.0625, 0.5625, 10.5625]]  # exact in binary


def test_equal_distances_across_subsets_order_by_row_id():
    # ids 1 and 2 lie at the same distance in different subsets; the lower id
    # comes first whichever subset holds it
    base = np.array([[0, 0], [3, 4], [4, 3], [10, 10], [-3, -4], [9, 9]], np.float32)
    q = np.zeros((1, 2), np.float32)
    for part in ([0, 0, 1, 1, 1, 0], [1, 1, 0, 0, 0, 1]):
        ids, d2 = oracle.partition_search(base, q, np.array(part), K=2, L_build=3, R=2, Cap=3, k=4, L=3)
        assert ids.tolist() == [[0, 1, 2, 4]]
        assert d2.tolist() == [[0.0, 25.0, 25.0, 25.0]]


def test_one_subset_is_the_plain_search():
    base, q = datagen.workload("tiny", n=800, nq=20)
    part = np.zeros(len(base), np.int32)
    ids, d2 = oracle.partition_search(base, q, part, K=12, L_build=30, R=10, Cap=60, k=10, L=40)
    g = oracle.build(base, 12, 30, 10, 60)
    rid, rd2, _, _ = oracle.search(g["adj"], base, g["nav"], q, 10, 40, deg=g["deg"])
    assert np.array_equal(ids, rid) and np.array_equal(d2, rd2)


@pytest.mark.parametrize("parts", [2, 3, 5])
def test_pool_covering_each_subset_gives_exact_knn(parts):
    # with L >= every subset's size each subset's search is its exact kNN
    # (every node is reachable after the connectivity pass), so the merge is
    # the exact kNN of the whole base
    base = datagen.uniform_int(600, 8, seed=11, hi=16)  # many distance ties
    q = datagen.uniform_int(30, 8, seed=12, hi=16)
    part = datagen.even_partition(len(base), parts, seed=parts)
    L = int(np.bincount(part).max())
    ids, d2 = oracle.partition_search(base, q, part, K=10, L_build=20, R=8, Cap=40, k=15, L=L)
    bid, bd2 = brute(base, q, 15)
    assert np.array_equal(d2.astype(np.float64), bd2)
    assert np.array_equal(ids, bid)


def test_fewer_rows_than_k_are_padded():
    base = np.array([[0.0], [1.0], [2.0], [3.0]], np.float32)
    part = np.array([0, 0, 1, 1])
    ids, d2 = oracle.partition_search(base, np.array([[0.5]], np.float32), part,
                                      K=1, L_build=2, R=1, Cap=2, k=6, L=6)
    assert ids.tolist() == [[0, 1, 2, 3, -1, -1]]
    assert np.isinf(d2[0, 4:]).all() and d2[0, :4].tolist() == [0.25, 0.25, 2.25, 6.25]


def test_rejects_bad_partitions():
    base = np.zeros((4, 2), np.float32)
    with pytest.raises(ValueError):
        oracle.partition_search(base, base[:1], np.array([0, 0, 1]), K=1, L_build=2, R=1, Cap=2, k=1, L=2)
    with pytest.raises(ValueError):
        oracle.partition_search(base, base[:1], np.array([0, 0, 0, 1]), K=1, L_build=2, R=1, Cap=2, k=1, L=2)
