"""Partition-and-merge search (Sections 4.2 and 4.3) against the oracle.

The base is split into random subsets, each gets its own Alg. 2 build, every
query runs Alg. 1 on every subset's graph and the union of the results is
cut to the k smallest (distance, row id) keys.  On integer data every
distance is exact, so the GPU path must equal the oracle bit for bit: each
subset's graph, and the merged ids and distances."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu

K, LB, R, CAP = 20, 40, 16, 200


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def tiny():
    return datagen.workload("tiny")


@pytest.mark.parametrize("P", [2, 3, 8])
def test_partitioned_search_bit_exact(nsg, tiny, P):
    base, q = tiny
    part = datagen.even_partition(len(base), P, seed=40 + P)
    idx = nsg.nsg_build_partitioned(T(base), part, K, LB, R, CAP, seed=0)
    assert idx.info()["parts"] == P
    for k, L in ((10, 50), (100, 120)):
        out = idx.search_partitioned(T(q), k, L)
        rid, rd2 = oracle.partition_search(base, q, part, K, LB, R, CAP, k, L, seed=0)
        assert np.array_equal(H(out["ids"]), rid), (P, k, L)
        assert np.array_equal(H(out["d2"]), rd2), (P, k, L)


def test_partitioned_graphs_equal_the_oracle_builds(nsg, tiny):
    base, _ = tiny
    P = 3
    part = datagen.even_partition(len(base), P, seed=7)
    idx = nsg.nsg_build_partitioned(T(base), part, K, LB, R, CAP, seed=0)
    adj, deg = (H(t) for t in idx.graph())
    off = 0
    for p in range(P):
        rows = np.flatnonzero(part == p)
        ref = oracle.build(base[rows], min(K, len(rows) - 1), LB, R, CAP, seed=0)
        sub = adj[off:off + len(rows)]
        assert np.array_equal(np.where(sub >= 0, sub - off, -1), ref["adj"]), p
        assert np.array_equal(deg[off:off + len(rows)], ref["deg"]), p
        off += len(rows)
    assert off == len(base)


def test_partitioned_precision_forms_and_small_subsets(nsg, tiny):
    # a subset smaller than k (padding of its list) and the 8-bit form, exact
    # on these values, give the same merged result
    base, q = tiny
    base = base[:3000]
    part = np.zeros(len(base), np.int32)
    part[1000:2995] = 1
    part[2995:] = 2  # 5 rows
    idx = nsg.nsg_build_partitioned(T(base), part, K, LB, R, CAP, seed=3)
    rid, rd2 = oracle.partition_search(base, q, part, K, LB, R, CAP, 10, 30, seed=3)
    out = idx.search_partitioned(T(q), 10, 30)
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)
    idx.prepare(nsg.PREC_U8)
    out = idx.search_partitioned(T(q), 10, 30, params=nsg.SearchParams(0, 0, nsg.PREC_U8, 0, -1))
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)


def test_partitioned_build_rejects_bad_partitions(nsg, tiny):
    base, _ = tiny
    base = base[:500]
    part = np.zeros(len(base), np.int32)
    part[-1] = 1  # a subset of one row
    with pytest.raises(nsg.NsgError) as e:
        nsg.nsg_build_partitioned(T(base), part, K, LB, R, CAP)
    assert e.value.status == nsg.NSG_EINVAL
    part[-1] = -1
    with pytest.raises(nsg.NsgError):
        nsg.nsg_build_partitioned(T(base), part, K, LB, R, CAP)
