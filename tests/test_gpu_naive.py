"""NSG-Naive (Section 4.1.2) on the GPU against the oracle: the MRNG
selection over the kNN graph's edges, and Alg. 1 with seeded random
initialisation (reading R10).  Integer data keeps every distance exact, so
graphs and search results must equal the oracle's bit for bit."""
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
def naive():
    base, q = datagen.workload("tiny", n=6000, nq=90)
    adj, deg = oracle.build_naive(base, 20, 16)
    return base, q, adj, deg


def test_build_naive_bit_exact(nsg, naive):
    base, _, adj, deg = naive
    idx = nsg.nsg_build_naive(T(base), 20, 16, seed=3)
    gadj, gdeg = idx.graph()
    assert np.array_equal(H(gdeg), deg)
    assert np.array_equal(H(gadj), adj)
    assert idx.info()["nav"] == oracle.splitmix64(3) % len(base)


@pytest.mark.parametrize("count,L,prec", [(1, 50, 0), (16, 50, 0), (50, 50, 0), (40, 100, 0), (40, 100, 3)])
def test_random_init_search_bit_exact(nsg, naive, count, L, prec):
    base, q, adj, deg = naive
    idx = nsg.nsg_index_from_graph(T(base), T(adj), 0, deg=T(deg))
    if prec:
        idx.prepare(prec)
    prm = nsg.SearchParams(0, 16384, prec, 0, -1, None, 0.5, 0, 0, count, 12345)
    out = idx.search_ex(T(q), 10, L, params=prm)
    rid, rd2, rne, rnd = oracle.search_random(adj, base, q, 10, L, count, 12345, deg=deg)
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)


def test_random_init_batched_equals_per_query(nsg, naive):
    base, q, adj, deg = naive
    idx = nsg.nsg_index_from_graph(T(base), T(adj), 0, deg=T(deg))
    k, L = datagen.uneven_k_L(len(q), seed=5, ks=(1, 10), l_lo=20, l_hi=120)
    prm = nsg.SearchParams(0, 0, 0, 0, -1, None, 0.5, 0, 0, 20, 99)
    out = idx.search_batched(T(q), T(k), T(L), params=prm)
    for i in range(0, len(q), 7):
        # query i draws from its own stream (its index in the batch), whatever
        # order the persistent warps take the queries in
        rid, _, _, _ = oracle.search_random(adj, base, q[:i + 1], int(k[i]), int(L[i]), 20, 99, deg=deg)
        assert H(out["ids"])[i, :k[i]].tolist() == rid[i].tolist()


def test_random_init_validation(nsg, naive):
    base, q, adj, deg = naive
    idx = nsg.nsg_index_from_graph(T(base), T(adj), 0, deg=T(deg))
    with pytest.raises(nsg.NsgError):
        idx.search_ex(T(q), 10, 20, params=nsg.SearchParams(0, 0, 0, 0, -1, None, 0.5, 0, 0, 21, 1))


def test_naive_recall_below_nsg(nsg):
    # the paper's point (Section 4.1.2): without search-collect, the navigating
    # node and connectivity, the same edge selection searches worse at equal L
    base, q = datagen.workload("tiny", n=8000, nq=100)
    gt, _ = oracle.knn_query(base, q, 10)
    nsg_idx = nsg.nsg_build(T(base), 20, 40, 16, 200, seed=0)
    naive_idx = nsg.nsg_build_naive(T(base), 20, 16, seed=0)
    a = H(nsg_idx.search(T(q), 10, 30)[0])
    b = H(naive_idx.search_ex(T(q), 10, 30, params=nsg.SearchParams(0, 0, 0, 0, -1, None, 0.5, 0, 0, 30, 1))["ids"])
    assert oracle.recall(a, gt, 10) > oracle.recall(b, gt, 10)
