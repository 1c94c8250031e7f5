"""Precision forms of the search: traversal distances on BF16 / FP8-e4m3 copies
of the base with FP32 accumulation, and an FP32 re-rank of the final pool.

Judged against the plain form and the oracle:
* integer data 0..255 is held exactly by BF16, so the BF16 form must equal
  the oracle bit for bit (with or without the re-rank);
* with re-rank, every returned distance is the exact FP32 squared distance
  of the returned id (checked against a float64 recomputation);
* FP8 traversal distances are within e4m3 rounding of the FP64 distances, and
  the re-ranked FP8 form loses at most 0.05 recall@10 against the plain form
  on these workloads (stated tolerance)."""
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
def tiny():
    base, q = datagen.workload("tiny", n=6000, nq=100)
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    gt, _ = oracle.knn_query(base, q, 10)
    return base, q, ref, gt


def _index(nsg, base, ref):
    return nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))


@pytest.mark.parametrize("rerank", [-1, 1])
def test_bf16_is_exact_on_integer_data(nsg, tiny, rerank):
    base, q, ref, _ = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_BF16)
    assert idx.info()["has_bf16"] == 2  # every value held exactly
    prm = nsg.SearchParams(0, 16384, nsg.PREC_BF16, 0, rerank)
    out = idx.search_ex(T(q), 10, 60, params=prm)
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, 10, 60, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)


def test_fp8_rerank_returns_exact_distances_and_bounded_recall_loss(nsg, tiny):
    base, q, ref, gt = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_FP8)
    info = idx.info()
    assert info["has_fp8"] >= 1 and abs(info["fp8_scale"] - 448.0 / base.max()) < 1e-6
    plain = idx.search_ex(T(q), 10, 60)
    fp8 = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, nsg.PREC_FP8, 0, 1))
    ids, d2 = H(fp8["ids"]), H(fp8["d2"])
    exact = ((base[ids].astype(np.float64) - q[:, None, :]) ** 2).sum(-1)
    assert np.array_equal(d2.astype(np.float64), exact)  # FP32 re-rank, exact on integer data
    for i in range(len(q)):  # sorted by (distance, id)
        keys = list(zip(d2[i].tolist(), ids[i].tolist()))
        assert keys == sorted(keys)
    r_plain = oracle.recall(H(plain["ids"]), gt, 10)
    r_fp8 = oracle.recall(ids, gt, 10)
    assert r_fp8 >= r_plain - 0.05


def test_fp8_traversal_distance_error_vs_fp64(nsg, tiny):
    base, q, ref, _ = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_FP8)
    s = idx.info()["fp8_scale"]
    out = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, nsg.PREC_FP8, 0, 0))
    ids, d2 = H(out["ids"]), H(out["d2"]).astype(np.float64) / (s * s)
    exact = ((base[ids].astype(np.float64) - q[:, None, :]) ** 2).sum(-1)
    rel = np.abs(d2 - exact) / np.maximum(exact, 1.0)
    # e4m3 keeps 3 mantissa bits: each coordinate is within 2^-4 relative, so a
    # squared difference of two such values can move by a few percent of |x|^2
    assert np.median(rel) < 0.1


def test_float_data_bf16_rerank(nsg):
    base = datagen.uniform_float(3000, 48, seed=81)
    q = datagen.uniform_float(80, 48, seed=82)
    ref = oracle.build(base, 16, 40, 14, 120, seed=1)
    gt, _ = oracle.knn_query(base, q, 10)
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_BF16)
    assert idx.info()["has_bf16"] == 1  # lossy on float data
    plain = idx.search_ex(T(q), 10, 80)
    lp = idx.search_ex(T(q), 10, 80, params=nsg.SearchParams(0, 0, nsg.PREC_BF16))  # auto: re-rank
    ids, d2 = H(lp["ids"]), H(lp["d2"])
    exact = ((base[ids].astype(np.float64) - q[:, None, :]) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-5, atol=0)
    assert oracle.recall(ids, gt, 10) >= oracle.recall(H(plain["ids"]), gt, 10) - 0.02


def test_precision_requires_prepare(nsg, tiny):
    base, q, ref, _ = tiny
    idx = _index(nsg, base, ref)
    with pytest.raises(nsg.NsgError) as e:
        idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, nsg.PREC_BF16))
    assert e.value.status == nsg.NSG_EINVAL
