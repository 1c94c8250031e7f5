"""Precision forms of the search: traversal distances on BF16 / FP8-e4m3 copies
of the base with FP32 accumulation or on an 8-bit copy with exact int32 sums,
and an FP32 re-rank of the final pool.

Checked against the plain form and the oracle:
* integer data 0..255 is held exactly by BF16, so the BF16 form must equal
  the oracle bit for bit (with or without the re-rank);
* with re-rank, every returned distance is the exact FP32 squared distance
  of the returned id (checked against a float64 recomputation);
* FP8 traversal distances are within e4m3 rounding of the FP64 distances, and
  the re-ranked FP8 form loses at most 0.05 recall@10 against the plain form
  on these workloads (stated tolerance);
* integer data spanning at most 256 values is held exactly by the 8-bit copy
  (x - min), so the U8 form equals the oracle bit for bit; queries the 8-bit
  map rounds, and lossy copies of float data, are re-ranked."""
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


@pytest.mark.parametrize("rerank", [-1, 0, 1])
def test_u8_is_exact_on_integer_data(nsg, tiny, rerank):
    # integer data of span <= 255: the 8-bit map is x - min, the int32 sums of
    # squared byte differences are the exact distances, so ids, distances and
    # the expansion counts equal the oracle's
    base, q, ref, _ = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_U8)
    info = idx.info()
    assert info["has_u8"] == 2 and info["u8_scale"] == 1.0 and info["u8_lo"] == base.min()
    prm = nsg.SearchParams(0, 16384, nsg.PREC_U8, 0, rerank)
    out = idx.search_ex(T(q), 10, 60, params=prm)
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, 10, 60, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)


def test_u8_offset_integer_data_is_exact(nsg):
    # signed integers: lo = min < 0 shifts both sides, differences unchanged
    rng = np.random.default_rng(83)
    base = (rng.integers(-120, 121, size=(2500, 40))).astype(np.float32)
    q = (rng.integers(-120, 121, size=(60, 40))).astype(np.float32)
    ref = oracle.build(base, 16, 40, 14, 120, seed=2)
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_U8)
    info = idx.info()
    assert info["has_u8"] == 2 and info["u8_lo"] == base.min() and info["u8_scale"] == 1.0
    out = idx.search_ex(T(q), 10, 50, params=nsg.SearchParams(0, 0, nsg.PREC_U8, 0, 0))
    rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 50, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)


def test_u8_rounded_queries_are_reranked(nsg, tiny):
    # the base is exact but these queries are not integers: the auto mode
    # re-ranks exactly those queries, so distances are FP32 ones of the ids
    base, q, ref, gt = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_U8)
    qf = q.astype(np.float32).copy()
    qf[::2] += 0.375  # every other query off the integer grid
    out = idx.search_ex(T(qf), 10, 60, params=nsg.SearchParams(0, 0, nsg.PREC_U8))
    ids, d2 = H(out["ids"]), H(out["d2"])
    exact = ((base[ids].astype(np.float64) - qf[:, None, :].astype(np.float64)) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-5, atol=0)
    plain = idx.search_ex(T(qf), 10, 60)
    gtf, _ = oracle.knn_query(base, qf, 10)
    assert oracle.recall(ids, gtf, 10) >= oracle.recall(H(plain["ids"]), gtf, 10) - 0.02


def test_u8_float_data_lossy_rerank(nsg):
    base = datagen.uniform_float(3000, 48, seed=84)
    q = datagen.uniform_float(80, 48, seed=85)
    ref = oracle.build(base, 16, 40, 14, 120, seed=1)
    gt, _ = oracle.knn_query(base, q, 10)
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_U8)
    info = idx.info()
    span = float(base.max()) - float(base.min())
    assert info["has_u8"] == 1 and abs(info["u8_scale"] - 255.0 / span) < 1e-6 * info["u8_scale"]
    plain = idx.search_ex(T(q), 10, 80)
    lp = idx.search_ex(T(q), 10, 80, params=nsg.SearchParams(0, 0, nsg.PREC_U8))  # auto: re-rank
    ids, d2 = H(lp["ids"]), H(lp["d2"])
    exact = ((base[ids].astype(np.float64) - q[:, None, :]) ** 2).sum(-1)
    assert np.allclose(d2, exact, rtol=1e-5, atol=0)
    assert oracle.recall(ids, gt, 10) >= oracle.recall(H(plain["ids"]), gt, 10) - 0.05


def test_rerank_list_outside_small_hash(nsg, tiny):
    # 64 hash slots hold 32 keys: k = 40 puts the re-rank list in its own region
    base, q, ref, _ = tiny
    idx = _index(nsg, base, ref)
    idx.prepare(nsg.PREC_BF16)
    for H_ in (64, 16384):
        out = idx.search_ex(T(q), 40, 60, params=nsg.SearchParams(0, H_, nsg.PREC_BF16, 0, 1))
        rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 40, 60, deg=ref["deg"])
        assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)
