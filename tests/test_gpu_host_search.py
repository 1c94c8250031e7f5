"""Search on host buffers (nsg_search_host): queries copied into staging the
index owns (grown on demand), one search launch, results copied back.
Results must equal the device-buffer search (nsg_search_ex) bit for bit --
for ragged batch sizes, page-locked or pageable host memory, with or without
distances, after the staging has grown -- and the oracle on integer data."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def sift20k(nsg):
    base, _ = datagen.workload("sift", n=20000, nq=1)
    idx = nsg.nsg_build(T(base), 20, 40, 24, 200, seed=0)
    return base, idx


@pytest.mark.parametrize("nq", [1, 37, 2047, 2048, 8191, 8192, 10001])
def test_host_search_equals_device_search(nsg, sift20k, nq):
    base, idx = sift20k
    q = datagen.uniform_int(nq, base.shape[1], seed=nq, hi=256)
    dev = idx.search_ex(T(q), 10, 64, counters=False)
    qh = torch.from_numpy(q).pin_memory()
    d2 = torch.empty((nq, 10), dtype=torch.float32).pin_memory()
    out = idx.search_host(qh, 10, 64, d2=d2)
    assert torch.equal(out["ids"], dev["ids"].cpu())
    assert torch.equal(out["d2"], dev["d2"].cpu())


def test_host_search_pageable_ids_only(nsg, sift20k):
    base, idx = sift20k
    q = datagen.uniform_int(3000, base.shape[1], seed=5, hi=256)
    dev = idx.search_ex(T(q), 16, 40, counters=False)
    out = idx.search_host(torch.from_numpy(q), 16, 40)
    assert out["d2"] is None
    assert torch.equal(out["ids"], dev["ids"].cpu())


def test_host_search_precision_form_and_growth(nsg, sift20k):
    # the 8-bit form through the host call; staging grows from earlier calls
    base, idx = sift20k
    idx.prepare(nsg.PREC_U8)
    prm = nsg.SearchParams(0, 0, nsg.PREC_U8)
    q = datagen.uniform_int(12000, base.shape[1], seed=6, hi=256)
    dev = idx.search_ex(T(q), 100, 150, params=prm, counters=False)
    out = idx.search_host(torch.from_numpy(q).pin_memory(), 100, 150, params=prm,
                          d2=torch.empty((12000, 100), dtype=torch.float32))
    assert torch.equal(out["ids"], dev["ids"].cpu())
    assert torch.equal(out["d2"], dev["d2"].cpu())


def test_host_search_equals_oracle(nsg):
    base, q = datagen.workload("tiny")
    ref = oracle.build(base, 20, 40, 16, 200, seed=0)
    idx = nsg.nsg_index_from_graph(T(base), T(ref["adj"]), ref["nav"])
    out = idx.search_host(torch.from_numpy(q), 10, 50, d2=torch.empty((len(q), 10), dtype=torch.float32))
    rid, rd2, _, _ = oracle.search(ref["adj"], base, ref["nav"], q, 10, 50, deg=ref["deg"])
    assert np.array_equal(out["ids"].numpy(), rid)
    assert np.array_equal(out["d2"].numpy(), rd2)


def test_host_search_step_cap_and_empty(nsg, sift20k):
    base, idx = sift20k
    q = datagen.uniform_int(50, base.shape[1], seed=7, hi=256)
    with pytest.raises(nsg.NsgError) as e:
        idx.search_host(torch.from_numpy(q), 10, 50, params=nsg.SearchParams(2, 0, nsg.PREC_F32, 0))
    assert e.value.status == nsg.NSG_ESTEPCAP
    out = idx.search_host(torch.empty((0, base.shape[1]), dtype=torch.float32), 10, 50)
    assert out["ids"].shape == (0, 10)
