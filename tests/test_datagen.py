"""The seeded input generators: shapes, value ranges, distributions, and the
chunked seeding that lets any row range regenerate on its own."""
import numpy as np
import pytest

from paper_1707_00143_gb300 import datagen


@pytest.mark.parametrize("name", sorted(datagen.WORKLOADS))
def test_prefix_and_row_ranges(name):
    mix = datagen.WORKLOADS[name]["mix"]
    whole = datagen.mixture_rows(mix, 1, 0, 70_000)  # spans two 65,536-row chunks
    assert whole.shape == (70_000, mix.d) and whole.dtype == np.float32
    part = datagen.mixture_rows(mix, 1, 65_000, 66_000)  # straddles the boundary
    assert np.array_equal(part, whole[65_000:66_000])
    base, q = datagen.workload(name, n=1000, nq=10)
    assert np.array_equal(base, whole[:1000])
    assert not np.array_equal(q, base[:10])  # queries come from their own seed


def test_value_ranges_and_distributions():
    s, _ = datagen.workload("sift", n=20_000, nq=1)
    assert (s == np.rint(s)).all() and s.min() >= 0 and s.max() <= 255
    g, _ = datagen.workload("gist", n=5_000, nq=1)
    assert g.min() >= 0 and g.max() <= 1
    d, _ = datagen.workload("deep", n=5_000, nq=1)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-5)
    r, _ = datagen.workload("rand4m", n=20_000, nq=1)
    assert r.min() >= 0 and r.max() < 1
    assert abs(r.mean() - 0.5) < 0.01 and abs(r.var() - 1 / 12) < 0.002  # U(0, 1)
    n, _ = datagen.workload("gauss5m", n=20_000, nq=1)
    assert abs(n.mean()) < 0.02 and abs(n.var() - 3.0) < 0.05  # N(0, 3), variance 3


def test_uneven_k_L():
    k, L = datagen.uneven_k_L(1000, seed=5, ks=(1, 10, 100), l_lo=20, l_hi=500)
    assert set(np.unique(k)) <= {1, 10, 100}
    assert (L >= k).all() and L.min() >= 20 and L.max() <= 500
