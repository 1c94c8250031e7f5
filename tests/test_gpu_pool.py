"""Pool placement: Alg. 1's pool of L keys in shared memory (L <= 1024) or in
a global-memory slot per resident warp (any L up to NSG_MAX_L).  Placement
changes where the keys live, not the steps: on integer data both must
reproduce the oracle's ids, distances and expansion counts bit for bit, at
pool sizes past the shared-memory limit too, and a batched plan mixing such
pool sizes returns every query's own fixed-(k, L) result."""
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
def setup(nsg):
    base, q = datagen.workload("tiny", n=10000, nq=120)
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    return base, q, ref, idx


@pytest.mark.parametrize("k,L", [(10, 1025), (100, 1500), (10, 3000)])
def test_large_pools_bit_exact(nsg, setup, k, L):
    base, q, ref, idx = setup
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, k, L, deg=ref["deg"],
                                       nthreads=oracle.nthreads_default())
    out = idx.search_ex(T(q), k, L, params=nsg.SearchParams(0, 16384, nsg.PREC_F32, 0))
    assert np.array_equal(H(out["ids"]), rid)
    assert np.array_equal(H(out["d2"]), rd2)
    assert np.array_equal(H(out["n_expand"]), rne)
    assert np.array_equal(H(out["n_dist"]), rnd)
    # the default (forgetful) visited set and the plain entry point
    ids, d2 = idx.search(T(q), k, L)
    assert np.array_equal(H(ids), rid) and np.array_equal(H(d2), rd2)
    # shared memory cannot hold these pools
    with pytest.raises(nsg.NsgError) as e:
        idx.search_ex(T(q), k, L, params=nsg.SearchParams(0, 0, nsg.PREC_F32, 0, pool=nsg.POOL_SHARED))
    assert e.value.status == nsg.NSG_EINVAL


@pytest.mark.parametrize("wpq", [1, 2, 4])
@pytest.mark.parametrize("prec", ["plain", "u8"])
def test_global_pool_equals_shared(nsg, setup, wpq, prec):
    base, q, ref, idx = setup
    p = {"plain": nsg.PREC_F32, "u8": nsg.PREC_U8}[prec]
    if p:
        idx.prepare(p)
    rid, rd2, rne, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 60, deg=ref["deg"])
    for pool in (nsg.POOL_SHARED, nsg.POOL_GLOBAL):
        prm = nsg.SearchParams(0, 0, p, 0, -1, None, 0.5, 0, 0, 0, 0, wpq, pool)
        out = idx.search_ex(T(q), 10, 60, params=prm)
        assert np.array_equal(H(out["ids"]), rid), pool
        assert np.array_equal(H(out["d2"]), rd2), pool
        assert np.array_equal(H(out["n_expand"]), rne), pool


def test_global_pool_trace_and_stop(nsg, setup):
    # the learned-stop and trace kernels take the global pool too
    base, q, ref, idx = setup
    prm = nsg.SearchParams(0, 16384, nsg.PREC_F32, 0, -1, None, 0.5, 10, 0, 0, 0, 1, nsg.POOL_GLOBAL)
    a = idx.search_trace(T(q[:5]), 10, 1200, 3000, params=prm)
    pools = [oracle.search_trace(ref["adj"], base, ref["nav"], q[i], 1200, max_steps=3000, deg=ref["deg"])
             for i in range(5)]
    assert [len(p) for p in pools] == H(a["steps"]).tolist()
    never = np.zeros(641, np.float16)
    never[640] = -30.0
    out = idx.search_ex(T(q), 10, 1200, params=nsg.SearchParams(0, 0, 0, 0, -1, T(never), 0.5, 10))
    rid, _, rne, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 1200, deg=ref["deg"])
    assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["n_expand"]), rne)


def test_batched_plan_mixing_pool_sizes(nsg, setup):
    base, q, ref, idx = setup
    k, L = datagen.uneven_k_L(len(q), seed=93, ks=(1, 10, 100), l_lo=20, l_hi=2000)
    assert (L > 1024).any() and (L <= 1024).any()
    plan = idx.plan(T(q), T(k), T(L), autotune=True)
    info = plan.info()
    assert info["pool"] == 2 and info["n_tried"] == 24  # only global pools hold L > 1024
    ids, d2 = plan.run()
    torch.cuda.synchronize()
    ids, d2 = H(ids), H(d2)
    for i in range(0, len(q), 7):
        rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q[i:i + 1], int(k[i]), int(L[i]),
                                       deg=ref["deg"])
        assert ids[i, :k[i]].tolist() == rid[0].tolist(), i
        assert np.array_equal(d2[i, :k[i]], rd2[0]), i
    out = idx.search_batched(T(q), T(k), T(L))
    assert np.array_equal(H(out["ids"]), ids)
