"""Staged row gathers: for rows of more than 512 values a warp can copy the
rows an expansion measures into a ring of shared-memory slots with the
bulk-copy (TMA) engine and measure them there, instead of loading a few rows
at a time into registers.  That changes how the rows reach the warp, not the
search (Alg. 1): on integer data every form must reproduce the oracle's ids,
distances and counters bit for bit with any ring size -- a ring of one slot,
rings smaller than an expansion's new rows (slots refilled while the warp
measures), the largest ring -- with one, two or four warps per query and
either pool placement; on float data the staged and register gathers give
the same keys, so the same results."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu

K_, L_ = 10, 64


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def wide(nsg):
    # GIST-wide integer rows (d = 960): FP32, BF16 and U8 distances are exact
    base = datagen.uniform_int(3000, 960, seed=81, hi=256)
    q = datagen.uniform_int(60, 960, seed=82, hi=256)
    ref = oracle.build(base, 16, 40, 24, 120, seed=0, nthreads=oracle.nthreads_default())
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    res = oracle.search(ref["adj"], base, ref["nav"], q, K_, L_, deg=ref["deg"], nthreads=oracle.nthreads_default())
    return base, q, ref, idx, res


def params(nsg, prec=0, stage=0, wpq=1, pool=0, hash_slots=16384):
    return nsg.SearchParams(0, hash_slots, prec, 0, -1, warps_per_query=wpq, pool=pool, stage_rows=stage)


def same(a, b):
    for key in ("ids", "d2", "n_expand", "n_dist"):
        assert torch.equal(a[key], b[key]), key


@pytest.mark.parametrize("wpq", [1, 2, 4])
@pytest.mark.parametrize("stage", [1, 3, 8, 32])
def test_staged_plain_bit_exact(nsg, wide, stage, wpq):
    base, q, ref, idx, (rid, rd2, rne, rnd) = wide
    out = idx.search_ex(T(q), K_, L_, params=params(nsg, 0, stage, wpq))
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)
    assert (H(out["status"]) == 0).all()


@pytest.mark.parametrize("prec", ["u8", "bf16", "fp8"])
@pytest.mark.parametrize("stage", [2, 32])
def test_staged_forms_equal_register(nsg, wide, prec, stage):
    # the traversal copy's rows staged, and the FP32 re-rank of the pool
    # gathered through the same ring (FP8 is lossy here: re-ranked)
    base, q, ref, idx, (rid, rd2, _, _) = wide
    p = {"u8": nsg.PREC_U8, "bf16": nsg.PREC_BF16, "fp8": nsg.PREC_FP8}[prec]
    idx.prepare(p)
    reg = idx.search_ex(T(q), K_, L_, params=params(nsg, p, -1))
    stg = idx.search_ex(T(q), K_, L_, params=params(nsg, p, stage))
    same(reg, stg)
    if prec != "fp8":  # exact copies: the oracle's own results
        assert np.array_equal(H(stg["ids"]), rid) and np.array_equal(H(stg["d2"]), rd2)


@pytest.mark.parametrize("wpq", [1, 4])
def test_staged_global_pool_and_large_L(nsg, wide, wpq):
    base, q, ref, idx, _ = wide
    L = 1100  # above what shared memory holds: the pools live in global memory
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q[:20], 100, L, deg=ref["deg"],
                                       nthreads=oracle.nthreads_default())
    out = idx.search_ex(T(q[:20]), 100, L, params=params(nsg, 0, 5, wpq))
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne) and np.array_equal(H(out["n_dist"]), rnd)
    shared = idx.search_ex(T(q), K_, L_, params=params(nsg, 0, 6, wpq, pool=nsg.POOL_SHARED))
    glob = idx.search_ex(T(q), K_, L_, params=params(nsg, 0, 6, wpq, pool=nsg.POOL_GLOBAL))
    same(shared, glob)


@pytest.mark.parametrize("d", [700, 1500])
def test_staged_float_rows(nsg, d):
    # float data, a width that pads (700 -> 704 floats) and the widest shape
    # (more than 1024 values): the staged keys are the register gather's keys
    base = datagen.uniform_float(1200, d, seed=83 + d)
    q = datagen.uniform_float(40, d, seed=84 + d)
    ref = oracle.build(base, 12, 30, 16, 80, seed=0, nthreads=oracle.nthreads_default())
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    reg = idx.search_ex(T(q), K_, 48, params=params(nsg, 0, -1))
    for stage in (2, 7):
        same(reg, idx.search_ex(T(q), K_, 48, params=params(nsg, 0, stage)))
    rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, K_, 48, deg=ref["deg"])
    got = H(reg["ids"])
    assert np.mean([len(set(got[i]) & set(rid[i])) / K_ for i in range(len(q))]) >= 0.999
    np.testing.assert_allclose(H(reg["d2"]), rd2, rtol=1e-5)


def test_staged_auto_plan_and_entry_points(nsg, wide):
    base, q, ref, idx, (rid, rd2, _, _) = wide
    # FP32 rows of 3,840 bytes: auto stages them (4 slots); warps per query
    # left to the library too
    auto = idx.search_ex(T(q), K_, L_, params=params(nsg, 0, 0))
    same(auto, idx.search_ex(T(q), K_, L_, params=params(nsg, 0, -1)))
    same(auto, idx.search_ex(T(q), K_, L_, params=params(nsg, 0, 0, wpq=0)))
    ids, d2 = idx.search(T(q), K_, L_)
    assert np.array_equal(H(ids), rid) and np.array_equal(H(d2), rd2)
    k, L = datagen.uneven_k_L(len(q), seed=85, ks=(1, 10), l_lo=20, l_hi=120)
    one = idx.search_batched(T(q), T(k), T(L), params=params(nsg, 0, -1, hash_slots=0))
    plan = idx.plan(T(q), T(k), T(L), autotune=True)
    pid, pd2 = plan.run()
    info = plan.info()
    assert info["stage_rows"] >= 0 and info["n_tried"] > 48  # the staged shapes were timed too
    assert torch.equal(pid, one["ids"]) and torch.equal(pd2, one["d2"])


def test_staged_validation(nsg, wide):
    base, q, ref, idx, _ = wide
    with pytest.raises(nsg.NsgError) as e:
        idx.search_ex(T(q), K_, L_, params=params(nsg, 0, nsg.STAGE_MAX + 1))
    assert e.value.status == nsg.NSG_EINVAL
    never = np.zeros(641, np.float16)
    never[640] = -30.0
    with pytest.raises(nsg.NsgError) as e:
        idx.search_ex(T(q), K_, L_, params=nsg.SearchParams(0, 0, 0, 0, -1, T(never), 0.5, 10, stage_rows=4))
    assert e.value.status == nsg.NSG_EINVAL
    small = datagen.uniform_int(500, 64, seed=86, hi=256)
    sref = oracle.build(small, 8, 20, 8, 40, seed=0)
    sidx = nsg.nsg_index_from_graph(T(small), T(sref["adj"]), sref["nav"], deg=T(sref["deg"]))
    with pytest.raises(nsg.NsgError) as e:  # rows of 512 values or fewer are never staged
        sidx.search_ex(T(small[:5]), 5, 20, params=params(nsg, 0, 4))
    assert e.value.status == nsg.NSG_EINVAL
