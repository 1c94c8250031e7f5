"""nsg_navigate_noalloc: the navigating-node search for callers that may not
allocate device memory (its visited bitmap is a fixed array inside the
library).  Its answer must equal nsg_navigate's, call after call, although
every call reuses the array the previous call left behind.  This file is
collected last so that a failure here never hides another test's result."""
import numpy as np
import pytest
import torch

from paper_1707_00143_gb300 import datagen

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_navigate_matches_allocating_entry_point(nsg):
    base, _ = datagen.workload("tiny", n=6000, nq=1)
    bt = T(base)
    knn, _ = nsg.nsg_knn_init(bt, 16)
    c = nsg.nsg_centroid(bt)
    for start, L in ((17, 40), (5999, 64)):  # two calls in a row: the second sees the first's leftovers
        ref = nsg.nsg_navigate(bt, knn, c, start, L)
        got = nsg.nsg_navigate_noalloc(bt, knn, c, start, L)
        assert got == ref
    # a smaller graph after a larger one: bits past its n are never read, cleared or not
    small = T(base[:700])
    kn2, _ = nsg.nsg_knn_init(small, 8)
    c2 = nsg.nsg_centroid(small)
    assert nsg.nsg_navigate_noalloc(small, kn2, c2, 3, 20) == nsg.nsg_navigate(small, kn2, c2, 3, 20)


def test_noalloc_navigate_rejects_oversized_and_bad_ids(nsg):
    import ctypes as C

    nav = C.c_int32(0)
    fake = C.c_void_p(256)  # never dereferenced: rejected before any launch
    assert nsg.lib().nsg_navigate_noalloc(fake, (1 << 24) + 1, 8, fake, 4, fake, 0, 10, C.byref(nav),
                                          None) == nsg.NSG_EINVAL
    base = datagen.uniform_int(300, 8, seed=71)
    knn = np.zeros((300, 4), np.int32)
    knn[5, 2] = 300  # out of range
    with pytest.raises(nsg.NsgError) as e:
        nsg.nsg_navigate_noalloc(T(base), T(knn), nsg.nsg_centroid(T(base)), 0, 10)
    assert e.value.status == nsg.NSG_EINVAL
