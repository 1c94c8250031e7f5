"""Brute-force kNN on the GPU (serial scan, Section 4.1.2) against the oracle.

Integer data in 0..255 with d <= 128 takes the tensor-core path (BF16 GEMM,
FP32 accumulation, fused top-k): distances are exact integers there, so ids
and distances must equal the oracle bit for bit.  Float data and rows wider
than 128 keep k + margin candidates by the GEMM distance and re-rank them
with exact FP32 distances; those differ from the oracle's only by summation
order (relative 1e-5, the tolerance stated for float data).  Rows wider than
1024 take the exact FP32 CUDA-core scan."""
import os

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


@pytest.fixture
def scan_engine():
    os.environ["NSG_KNN_ENGINE"] = "scan"
    yield
    os.environ.pop("NSG_KNN_ENGINE", None)


@pytest.mark.parametrize("n,d,k,hi", [(1000, 32, 10, 256), (777, 128, 100, 256), (2000, 96, 256, 256),
                                      (1300, 64, 17, 3), (300, 128, 1, 256)])
def test_knn_init_tensor_core_bit_exact(nsg, n, d, k, hi):
    # ragged row blocks (n % 128 != 0), K padding (d = 96 -> 128), ties (hi = 3)
    base = datagen.uniform_int(n, d, seed=n + d, hi=hi)
    ids, d2 = nsg.nsg_knn_init(T(base), k)
    rid, rd2 = oracle.knn_rows(base, k)
    assert np.array_equal(H(d2), rd2)
    assert np.array_equal(H(ids), rid)


@pytest.mark.parametrize("nq,k", [(1, 10), (129, 100), (300, 256)])
def test_knn_query_tensor_core_bit_exact(nsg, nq, k):
    base, q = datagen.workload("tiny", n=5000, nq=nq)
    ids, d2 = nsg.nsg_knn_query(T(base), T(q), k)
    rid, rd2 = oracle.knn_query(base, q, k)
    assert np.array_equal(H(d2), rd2)
    assert np.array_equal(H(ids), rid)


def test_tensor_core_equals_scan_engine(nsg, scan_engine):
    base = datagen.duplicate_rows(datagen.uniform_int(3000, 128, seed=61, hi=8), 200, seed=62)
    a_ids, a_d2 = nsg.nsg_knn_init(T(base), 50)  # scan (fixture sets the engine)
    os.environ.pop("NSG_KNN_ENGINE")
    b_ids, b_d2 = nsg.nsg_knn_init(T(base), 50)  # tensor cores
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d2, b_d2)


def test_float_data_uses_exact_scan_within_tolerance(nsg):
    base = datagen.uniform_float(2500, 40, seed=63)
    q = datagen.uniform_float(70, 40, seed=64)
    ids, d2 = nsg.nsg_knn_query(T(base), T(q), 20)
    rid, rd2 = oracle.knn_query(base, q, 20)
    ids, d2 = H(ids), H(d2)
    assert np.allclose(d2, rd2, rtol=1e-5, atol=0)
    # ids agree except where two candidates are within rounding of each other
    same = (ids == rid).mean()
    assert same > 0.99
    exact = ((base[ids].astype(np.float64) - q[:, None, :]) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-5, atol=0)


def test_knn_large_d_bit_exact(nsg):
    # d = 200 > 128: the streaming tensor-core form (64-wide K chunks) keeps
    # candidates, the FP32 re-rank picks the k; integer data is exact in any order
    base = datagen.uniform_int(900, 200, seed=65)
    ids, d2 = nsg.nsg_knn_init(T(base), 30)
    rid, rd2 = oracle.knn_rows(base, 30)
    assert np.array_equal(H(ids), rid) and np.array_equal(H(d2), rd2)


def test_knn_init_ids_only(nsg):
    # the build asks for ids only; the tensor-core path keeps its lists in scratch then
    base = datagen.uniform_int(1500, 64, seed=66)
    ids, d2 = nsg.nsg_knn_init(T(base), 20, with_d2=False)
    assert d2 is None
    rid, _ = oracle.knn_rows(base, 20)
    assert np.array_equal(H(ids), rid)


@pytest.mark.parametrize("n,d,k", [(2000, 960, 100), (1500, 1024, 10), (900, 1028, 20)])
def test_knn_wide_float_rows(nsg, n, d, k):
    base = datagen.uniform_float(n, d, seed=d)
    ids, d2 = nsg.nsg_knn_init(T(base), k)
    rid, rd2 = oracle.knn_rows(base, k)
    ids, d2 = H(ids), H(d2)
    assert np.allclose(d2, rd2, rtol=1e-5, atol=0)
    exact = ((base[ids].astype(np.float64) - base[:, None, :]) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-5, atol=0)
    # ids may swap only among near-ties: none is farther than the true k-th
    # distance beyond rounding, and the sets agree
    assert (exact <= rd2[:, -1:].astype(np.float64) * (1 + 1e-5)).all()
    assert oracle.recall(ids, rid, k) >= 0.995
    # and every row is a valid answer: k distinct existing rows, never itself,
    # in ascending distance -- with the bound above, k rows none of which is
    # farther than the true k-th neighbour
    assert ((ids >= 0) & (ids < n)).all()
    assert all(len(set(row.tolist())) == k for row in ids)
    assert not (ids == np.arange(n)[:, None]).any()
    assert (np.diff(d2, axis=1) >= 0).all()


def test_knn_query_gist_shaped(nsg):
    base, q = datagen.workload("gist", n=4000, nq=64)
    ids, d2 = nsg.nsg_knn_query(T(base), T(q), 100)
    rid, rd2 = oracle.knn_query(base, q, 100)
    assert np.allclose(H(d2), rd2, rtol=1e-5, atol=0)
    assert oracle.recall(H(ids), rid, 100) >= 0.999


def test_knn_deep_shaped_unit_norm(nsg):
    base, _ = datagen.workload("deep", n=5000, nq=1)
    ids, d2 = nsg.nsg_knn_init(T(base), 64)
    rid, rd2 = oracle.knn_rows(base, 64)
    assert np.allclose(H(d2), rd2, rtol=1e-5, atol=1e-7)
    assert oracle.recall(H(ids), rid, 64) >= 0.999


@pytest.fixture
def small_chunks():
    # the tensor-core kNN takes the base in chunks (one launch each) and
    # carries every row's list across them; 3-tile chunks exercise that here
    os.environ["NSG_KNN_CHUNK_TILES"] = "3"
    yield
    os.environ.pop("NSG_KNN_CHUNK_TILES", None)


@pytest.mark.parametrize("n,d,k,hi", [(1000, 32, 10, 256), (1300, 128, 100, 3), (700, 128, 256, 256)])
def test_knn_chunked_base_bit_exact(nsg, small_chunks, n, d, k, hi):
    base = datagen.uniform_int(n, d, seed=n + 7 * d, hi=hi)
    ids, d2 = nsg.nsg_knn_init(T(base), k)
    rid, rd2 = oracle.knn_rows(base, k)
    assert np.array_equal(H(d2), rd2) and np.array_equal(H(ids), rid)
    q = datagen.uniform_int(150, d, seed=n + 1, hi=hi)
    ids, d2 = nsg.nsg_knn_query(T(base), T(q), k)
    rid, rd2 = oracle.knn_query(base, q, k)
    assert np.array_equal(H(d2), rd2) and np.array_equal(H(ids), rid)


def test_knn_chunked_float_rerank(nsg, small_chunks):
    base = datagen.uniform_float(1500, 200, seed=67)
    ids, d2 = nsg.nsg_knn_init(T(base), 20)
    rid, rd2 = oracle.knn_rows(base, 20)
    ids, d2 = H(ids), H(d2)
    assert np.allclose(d2, rd2, rtol=1e-5, atol=0)
    exact = ((base[ids].astype(np.float64) - base[:, None, :]) ** 2).sum(-1)
    assert (exact <= rd2[:, -1:].astype(np.float64) * (1 + 1e-5)).all()
    assert oracle.recall(ids, rid, 20) >= 0.995
