"""Several warps per query (warps_per_query 2 or 4): the leader warp expands,
every warp measures a slice of the new neighbours, the leader merges.  The
steps are Alg. 1's, so results, expansion and distance counts must equal the
one-warp search and the oracle bit for bit on integer data."""
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
    base, q = datagen.workload("tiny", n=8000, nq=150)
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    return base, q, ref


@pytest.mark.parametrize("wpq", [2, 4])
@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("wpc", [0, 8])
def test_group_search_equals_oracle(nsg, tiny, wpq, prec, wpc):
    base, q, ref = tiny
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    if prec:
        idx.prepare(prec)
    prm = nsg.SearchParams(0, 16384, prec, wpc, -1, warps_per_query=wpq)
    out = idx.search_ex(T(q), 10, 70, params=prm)
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, 10, 70, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)
    assert (H(out["status"]) == 0).all()


@pytest.mark.parametrize("wpq", [2, 4])
def test_group_random_init_and_default_hash(nsg, tiny, wpq):
    base, q, ref = tiny
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    one = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, 0, 0, -1, None, 0.5, 0, 0, 25, 3,
                                                              warps_per_query=1))
    grp = idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(0, 0, 0, 0, -1, None, 0.5, 0, 0, 25, 3,
                                                              warps_per_query=wpq))
    assert torch.equal(one["ids"], grp["ids"]) and torch.equal(one["d2"], grp["d2"])
    assert torch.equal(one["n_expand"], grp["n_expand"])


@pytest.mark.parametrize("wpq", [2, 4])
def test_group_wide_rows_and_step_cap(nsg, wpq):
    base = datagen.uniform_int(2000, 600, seed=7, hi=64)
    q = datagen.uniform_int(40, 600, seed=8, hi=64)
    ref = oracle.build(base, 12, 30, 12, 100, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    out = idx.search_ex(T(q), 10, 48, params=nsg.SearchParams(0, 16384, 0, 0, -1, warps_per_query=wpq))
    rid, rd2, rne, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 48, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    capped = idx.search_ex(T(q), 10, 48, params=nsg.SearchParams(5, 0, 0, 0, -1, warps_per_query=wpq))
    assert (H(capped["status"]) == nsg.NSG_ESTEPCAP).all() and (H(capped["n_expand"]) == 5).all()


def test_group_batched_and_validation(nsg, tiny):
    base, q, ref = tiny
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    k, L = datagen.uneven_k_L(len(q), seed=9, ks=(1, 10, 50), l_lo=20, l_hi=150)
    one = idx.search_batched(T(q), T(k), T(L), params=nsg.SearchParams(warps_per_query=1))
    grp = idx.search_batched(T(q), T(k), T(L), params=nsg.SearchParams(warps_per_query=4))
    auto = idx.search_batched(T(q), T(k), T(L))  # warps per query left to the library
    assert torch.equal(one["ids"], auto["ids"]) and torch.equal(one["d2"], auto["d2"])
    assert torch.equal(one["ids"], grp["ids"]) and torch.equal(one["d2"], grp["d2"])
    with pytest.raises(nsg.NsgError):
        idx.search_ex(T(q), 10, 60, params=nsg.SearchParams(warps_per_query=3))
