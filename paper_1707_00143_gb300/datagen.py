"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the CUDA path, the CPU oracle and the
tests.  It draws random numbers and nothing else: no distance, no search, no
graph arithmetic lives here.

The paper's datasets (SIFT1M, GIST1M, DEEP100M; Table 1 of Section 4.1) are
not available, so each workload is a Gaussian mixture with the dimension, size
and value range of the dataset it stands in for:

* ``tiny``   10,000 x 32, integer values 0..255, 16 components, sigma 30,
             100 queries (small parity case).
* ``sift``   1,000,000 x 128, integer values 0..255, 100 components, sigma 30,
             10,000 queries (SIFT1M shape: D=128, integer 0..255).
* ``gist``   1,000,000 x 960, floats in [0, 1], 50 components, sigma 0.1,
             1,000 queries (GIST1M shape: D=960, real values).
* ``deep``   10,000,000 x 96, unit-norm floats, 1,000 components, sigma 0.05,
             100,000 queries (DEEP shape: D=96).
* ``rand4m`` 4,000,000 x 128, i.i.d. U(0, 1) coordinates, 10,000 queries (the
             paper's RAND4M, Section 4.1.1).
* ``gauss5m`` 5,000,000 x 128, i.i.d. N(0, 3) coordinates, read as variance 3
             (standard deviation sqrt(3)), 10,000 queries (the paper's GAUSS5M;
             a common scale factor changes no distance order, so the other
             reading, sigma = 3, gives the same graph and results).

Rows are generated in fixed-size chunks, each from its own generator seeded
by ``(seed, chunk_index)``, so any row range can be regenerated on its own and
the result does not depend on how the caller slices the work.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

CHUNK = 65536


@dataclass(frozen=True)
class Mixture:
    """A Gaussian-mixture recipe for one workload."""

    d: int
    n_components: int
    sigma: float
    kind: str               # "int255" | "unit01" | "unitnorm" | "uniform01" | "gauss"
    centre_lo: float = 0.0
    centre_hi: float = 1.0
    seed_centres: int = 3


WORKLOADS = {
    "tiny": dict(mix=Mixture(32, 16, 30.0, "int255", 40.0, 215.0), n=10_000, nq=100),
    "sift": dict(mix=Mixture(128, 100, 30.0, "int255", 40.0, 215.0), n=1_000_000, nq=10_000),
    "gist": dict(mix=Mixture(960, 50, 0.1, "unit01", 0.2, 0.8), n=1_000_000, nq=1_000),
    "deep": dict(mix=Mixture(96, 1000, 0.05, "unitnorm"), n=10_000_000, nq=100_000),
    "rand4m": dict(mix=Mixture(128, 1, 0.0, "uniform01"), n=4_000_000, nq=10_000),
    "gauss5m": dict(mix=Mixture(128, 1, 3.0 ** 0.5, "gauss"), n=5_000_000, nq=10_000),
}

SEED_BASE = 1
SEED_QUERY = 2


def centres(mix: Mixture) -> np.ndarray:
    rng = np.random.default_rng(mix.seed_centres)
    if mix.kind == "unitnorm":
        c = rng.standard_normal((mix.n_components, mix.d))
        c /= np.linalg.norm(c, axis=1, keepdims=True)
        return c
    return rng.uniform(mix.centre_lo, mix.centre_hi, size=(mix.n_components, mix.d))


def _chunk(mix: Mixture, cen: np.ndarray, seed: int, chunk: int, rows: int) -> np.ndarray:
    rng = np.random.default_rng([seed, chunk])
    if mix.kind == "uniform01":  # i.i.d. coordinates, no mixture
        return rng.random((rows, mix.d), dtype=np.float64).astype(np.float32)
    if mix.kind == "gauss":
        return rng.normal(0.0, mix.sigma, size=(rows, mix.d)).astype(np.float32)
    comp = rng.integers(0, mix.n_components, size=rows)
    x = cen[comp] + rng.normal(0.0, mix.sigma, size=(rows, mix.d))
    if mix.kind == "int255":
        x = np.clip(np.rint(x), 0.0, 255.0)
    elif mix.kind == "unit01":
        x = np.clip(x, 0.0, 1.0)
    elif mix.kind == "unitnorm":
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32)


def mixture_rows(mix: Mixture, seed: int, start: int, stop: int) -> np.ndarray:
    """Rows ``start..stop`` of the stream drawn with ``seed`` (float32 [rows][d])."""
    out = np.empty((max(stop - start, 0), mix.d), dtype=np.float32)
    if stop <= start:
        return out
    cen = centres(mix)
    for c in range(start // CHUNK, (stop - 1) // CHUNK + 1):
        lo, hi = c * CHUNK, (c + 1) * CHUNK
        blk = _chunk(mix, cen, seed, c, CHUNK)
        a, b = max(lo, start), min(hi, stop)
        out[a - start:b - start] = blk[a - lo:b - lo]
    return out


def workload(name: str, n: int | None = None, nq: int | None = None,
             seed_base: int = SEED_BASE, seed_query: int = SEED_QUERY):
    """(base [n][d], queries [nq][d]) float32 for a named workload.

    ``n`` / ``nq`` override the sizes (a prefix of the same stream)."""
    w = WORKLOADS[name]
    mix = w["mix"]
    n = w["n"] if n is None else n
    nq = w["nq"] if nq is None else nq
    return mixture_rows(mix, seed_base, 0, n), mixture_rows(mix, seed_query, 0, nq)


def uniform_int(n: int, d: int, seed: int, hi: int = 256) -> np.ndarray:
    """Uniform integers 0..hi-1 stored as float32 (many exact distance ties when hi is small)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(n, d)).astype(np.float32)


def uniform_float(n: int, d: int, seed: int) -> np.ndarray:
    """Uniform floats in [0, 1) (general position: ties have probability zero)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, d), dtype=np.float64).astype(np.float32)


def duplicate_rows(x: np.ndarray, n_dup: int, seed: int) -> np.ndarray:
    """Copy ``n_dup`` random rows over other random rows (exact duplicate points)."""
    rng = np.random.default_rng(seed)
    y = x.copy()
    src = rng.integers(0, len(x), size=n_dup)
    dst = rng.integers(0, len(x), size=n_dup)
    y[dst] = x[src]
    return y


def uneven_k_L(nq: int, seed: int, ks=(1, 10, 100), l_lo: int = 20, l_hi: int = 500):
    """Per-query (k, L) for the batched uneven-query workload: k from ``ks``,
    L uniform in [l_lo, l_hi], then L raised to at least k."""
    rng = np.random.default_rng(seed)
    k = rng.choice(np.asarray(ks, dtype=np.int32), size=nq).astype(np.int32)
    L = rng.integers(l_lo, l_hi + 1, size=nq).astype(np.int32)
    return k, np.maximum(L, k).astype(np.int32)


def even_partition(n: int, parts: int, seed: int) -> np.ndarray:
    """Random even split of rows 0..n-1 into ``parts`` subsets (the partition
    of the partitioned search of Sections 4.2 and 4.3): a seeded permutation dealt out in
    turn, so subset sizes differ by at most one.  Returns int32 [n] subset ids."""
    rng = np.random.default_rng(seed)
    part = np.empty(n, np.int32)
    part[rng.permutation(n)] = np.arange(n, dtype=np.int64) % parts
    return part
