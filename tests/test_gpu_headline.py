"""The benchmark's search configuration against the oracle, element by element.

The SIFT-shaped benchmark searches an index built at K=100, L=40, R=50,
C=500 with k=100 results from a pool of L=138, in the launch shape the
benchmark times (default visited set of 512 slots, default warps per block,
the device work counter).  At R=50 every expansion reads its adjacency row in
two 32-slot rounds and merges up to 50 new keys, a path the 16-wide tiny
graphs never take.  Here a 20,000-row base of the same recipe is built by the
oracle (Alg. 2) and searched (Alg. 1, Section 3.6) by both sides: on integer
data every float32 squared distance is exact, so ids, distances and expansion
counts must agree bit for bit, for the plain, BF16 and 8-bit forms and for
1, 2 and 4 warps per query.

R=220 (the degree the paper's high-LID synthetic sets reach, Table 2) takes
the adjacency loop past 128 slots; it is checked on integer rows (bit-exact)
and on i.i.d. U(0,1) float rows (distances to 1e-5 relative, recall against
the oracle's ids within 0.001)."""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu

K, LB, R, CAP = 100, 40, 50, 500  # the SIFT-shaped build
KQ, LQ = 100, 138  # the benchmark's operating point


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def H(t):
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def sift20k():
    base, q = datagen.workload("sift", n=20000, nq=300)
    ref = oracle.build(base, K, LB, R, CAP, seed=0)
    rid, rd2, rne, rnd = oracle.search(ref["adj"], base, ref["nav"], q, KQ, LQ, deg=ref["deg"],
                                       nthreads=oracle.nthreads_default())
    return dict(base=base, q=q, ref=ref, rid=rid, rd2=rd2, rne=rne, rnd=rnd)


def test_headline_build_bit_exact(nsg, sift20k):
    # the GPU build at the benchmark's build parameters equals the oracle's graph
    base, ref = sift20k["base"], sift20k["ref"]
    idx = nsg.nsg_build(T(base), K, LB, R, CAP, seed=0)
    adj, deg = idx.graph()
    assert idx.info()["nav"] == ref["nav"]
    assert np.array_equal(H(deg), ref["deg"])
    assert np.array_equal(H(adj), ref["adj"])
    assert ref["deg"].max() > 32  # rows span two 32-slot rounds


@pytest.mark.parametrize("form", ["plain", "bf16", "u8"])
@pytest.mark.parametrize("wpq", [1, 2, 4])
def test_headline_search_bit_exact(nsg, sift20k, form, wpq):
    base, q, ref = sift20k["base"], sift20k["q"], sift20k["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    prec = {"plain": nsg.PREC_F32, "bf16": nsg.PREC_BF16, "u8": nsg.PREC_U8}[form]
    if prec != nsg.PREC_F32:
        idx.prepare(prec)
        assert idx.info()["has_" + form] == 2  # exact copy on 0..255 data: no re-rank
    # the benchmark's parameters: default visited set, default warps per block
    params = nsg.SearchParams(0, 0, prec, 0, -1, None, 0.5, 0, 0, 0, 0, wpq)
    out = idx.search_ex(T(q), KQ, LQ, params=params)
    assert np.array_equal(H(out["ids"]), sift20k["rid"])
    assert np.array_equal(H(out["d2"]), sift20k["rd2"])
    assert np.array_equal(H(out["n_expand"]), sift20k["rne"])
    # the 512-slot set may forget a node and measure it again: never fewer
    assert (H(out["n_dist"]) >= sift20k["rnd"]).all()
    assert (H(out["status"]) == 0).all()
    # an exact visited set and 8 warps per block reproduce the distance counts too
    exact = nsg.SearchParams(0, 16384, prec, 8, -1, None, 0.5, 0, 0, 0, 0, wpq)
    out = idx.search_ex(T(q), KQ, LQ, params=exact)
    assert np.array_equal(H(out["ids"]), sift20k["rid"])
    assert np.array_equal(H(out["n_expand"]), sift20k["rne"])
    assert np.array_equal(H(out["n_dist"]), sift20k["rnd"])


def test_headline_host_buffer_search(nsg, sift20k):
    # the end-to-end call of the benchmark (host buffers in and out)
    base, q, ref = sift20k["base"], sift20k["q"], sift20k["ref"]
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"], deg=T(ref["deg"]))
    idx.prepare(nsg.PREC_U8)
    qh = torch.from_numpy(q).pin_memory()
    got = idx.search_host(qh, KQ, LQ, params=nsg.SearchParams(0, 0, nsg.PREC_U8, 0, -1))
    assert np.array_equal(got["ids"].numpy(), sift20k["rid"])


@functools.lru_cache(maxsize=None)
def _wide_case(kind):
    n, d, nq = 5000, 128, 120
    if kind == "int":
        base = datagen.uniform_int(n, d, seed=220, hi=256)
        q = datagen.uniform_int(nq, d, seed=221, hi=256)
    else:
        base, q = datagen.workload("rand4m", n=n, nq=nq)
    ref = oracle.build(base, 150, 150, 220, 500, seed=0)
    return base, q, ref


def _random_wide_graph(n, width, seed):
    # every row lists 129..width distinct random neighbours (no self loop):
    # each expansion reads ids past slot 128
    rng = np.random.default_rng(seed)
    adj = np.full((n, width), -1, np.int32)
    deg = rng.integers(129, width + 1, n).astype(np.int32)
    for v in range(n):
        row = rng.choice(n - 1, deg[v], replace=False)
        row[row >= v] += 1
        adj[v, :deg[v]] = row
    return adj, deg


@pytest.mark.parametrize("kind", ["int", "float"])
@pytest.mark.parametrize("graph", ["nsg", "random"])
def test_r220_search(nsg, kind, graph):
    base, q, ref = _wide_case(kind)
    if graph == "nsg":
        adj, deg, nav = ref["adj"], ref["deg"], ref["nav"]
        assert (deg > 128).sum() >= 5  # rows with neighbours past slot 128
    else:
        adj, deg = _random_wide_graph(len(base), 220, seed=222)
        nav = 0
    assert adj.shape[1] == 220
    idx = nsg.nsg_index_from_graph(T(base), T(adj), nav, deg=T(deg))
    k, L = 10, 120
    rid, rd2, rne, rnd = oracle.search(adj, base, nav, q, k, L, deg=deg)
    out = idx.search_ex(T(q), k, L, params=nsg.SearchParams(0, 16384, nsg.PREC_F32, 0))
    ids, d2 = H(out["ids"]), H(out["d2"])
    if kind == "int":
        assert np.array_equal(ids, rid)
        assert np.array_equal(d2, rd2)
        assert np.array_equal(H(out["n_expand"]), rne)
        # ~5,000 distances per query on the random graph can overflow a bucket
        # of the 16,384-slot set (then a node is measured twice); not on the NSG
        if graph == "nsg":
            assert np.array_equal(H(out["n_dist"]), rnd)
        else:
            assert (H(out["n_dist"]) >= rnd).all()
        # default visited set, and the 8-bit form: same results
        out = idx.search_ex(T(q), k, L)
        assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["n_expand"]), rne)
        idx.prepare(nsg.PREC_U8)
        out = idx.search_ex(T(q), k, L, params=nsg.SearchParams(0, 0, nsg.PREC_U8, 0, -1))
        assert np.array_equal(H(out["ids"]), rid) and np.array_equal(H(out["n_expand"]), rne)
    else:
        assert np.allclose(d2, rd2, rtol=1e-5, atol=0)
        assert oracle.recall(ids, rid, k) >= 1.0 - 0.001


def test_r220_build_bit_exact(nsg):
    base, _, ref = _wide_case("int")
    idx = nsg.nsg_build(T(base), 150, 150, 220, 500, seed=0)
    adj, deg = idx.graph()
    assert idx.info()["nav"] == ref["nav"]
    assert np.array_equal(H(deg), ref["deg"])
    assert np.array_equal(H(adj), ref["adj"])
