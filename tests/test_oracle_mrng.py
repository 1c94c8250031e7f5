"""Oracle pins for the MRNG edge selection (Def. MRNG, Sec. 3.3, Lemma 1/2, Thm 3)."""
import os

import numpy as np
import pytest

import oracle
from checkers import (edges_of, msnet_violations, mrng_fixpoint_violations,
                      occlusion_violations, read_golden, sqdist_matrix)
from paper_1707_00143_gb300 import datagen


def _golden_cases(golden_dir):
    cases, cur = [], None
    for tag, v in read_golden(os.path.join(golden_dir, "mrng_small.txt")):
        if tag == "case":
            cur = dict(pts={})
            cases.append(cur)
        elif tag == "point":
            cur["pts"][int(v[0])] = [float(v[1]), float(v[2])]
        elif tag == "node":
            cur["node"] = int(v[0])
        else:
            cur[tag] = [int(x) for x in v]
    return cases


def test_prune_hand_examples(golden_dir):
    for c in _golden_cases(golden_dir):
        n = len(c["pts"])
        base = np.array([c["pts"][i] for i in range(n)], np.float32)
        p = c["node"]
        D = sqdist_matrix(base, base)[p]
        others = sorted((D[q], q) for q in range(n) if q != p)
        ids = np.array([q for _, q in others], np.int32)
        dist = np.array([d for d, _ in others], np.float32)
        row, deg = oracle.prune(base, ids, dist, n)
        assert row[:deg].tolist() == c["kept_uncapped"]
        row, deg = oracle.prune(base, ids, dist, 2)
        assert row[:deg].tolist() == c["kept_R2"]


@pytest.mark.parametrize("d,seed", [(2, 31), (3, 32), (5, 33)])
def test_naive_mrng_satisfies_definition_and_lemma1(d, seed):
    base = datagen.uniform_float(45, d, seed=seed)
    adj, deg = oracle.mrng_naive(base)
    E = edges_of(adj, deg)
    assert mrng_fixpoint_violations(base, E) == []  # Def. MRNG
    assert msnet_violations(base, E) == []  # Thm 3 via Lemma 1


def test_naive_mrng_on_integer_ties_satisfies_definition():
    base = datagen.uniform_int(40, 2, seed=34, hi=6)
    base = np.unique(base, axis=0)  # distinct points; many equal distances remain
    adj, deg = oracle.mrng_naive(base)
    assert mrng_fixpoint_violations(base, edges_of(adj, deg)) == []


def test_checkers_reject_planted_mistakes():
    # the definition checker must notice a dropped edge and an occluded edge
    base = datagen.uniform_float(30, 2, seed=35)
    adj, deg = oracle.mrng_naive(base)
    E = edges_of(adj, deg)
    dropped = [list(e) for e in E]
    victim = max(range(30), key=lambda p: len(E[p]))
    dropped[victim] = dropped[victim][:-1]
    assert mrng_fixpoint_violations(base, dropped)
    added = [list(e) for e in E]
    D = sqdist_matrix(base, base)
    p = 0
    extra = next(q for q in np.argsort(D[p]) if q != p and q not in added[p])
    added[p].append(int(extra))
    assert mrng_fixpoint_violations(base, added)
    # a graph without the nearest-neighbour edges is not an MSNET
    nonn = [e[1:] for e in E]
    assert msnet_violations(base, nonn)


def test_mrng_contains_nng_and_60_degree_rule():
    base = datagen.uniform_float(60, 4, seed=36)
    adj, deg = oracle.mrng_naive(base)
    D = sqdist_matrix(base, base)
    np.fill_diagonal(D, np.inf)
    nn = np.argmin(D, axis=1)
    for p in range(60):
        assert nn[p] in adj[p][: deg[p]]  # NNG subset of MRNG (Sec. 3.3)
    assert occlusion_violations(base, adj, deg) == []
    # Lemma 2's argument: any two edges from p make an angle >= 60 degrees
    X = base.astype(np.float64)
    for p in range(60):
        row = adj[p][: deg[p]]
        for a in range(len(row)):
            for b in range(a):
                u, v = X[row[a]] - X[p], X[row[b]] - X[p]
                cos = u @ v / np.sqrt((u @ u) * (v @ v))
                assert cos <= 0.5 + 1e-6


def test_prune_cap_is_prefix_of_uncapped():
    base = datagen.uniform_float(80, 3, seed=37)
    D = sqdist_matrix(base, base)
    for p in range(0, 80, 7):
        order = sorted((D[p, q], q) for q in range(80) if q != p)
        ids = np.array([q for _, q in order], np.int32)
        dist = np.array([d for d, _ in order], np.float32)
        full, dfull = oracle.prune(base, ids, dist, 79)
        for R in (1, 2, 3, 5):
            row, dg = oracle.prune(base, ids, dist, R)
            assert dg == min(R, dfull)
            assert row[:dg].tolist() == full[:dg].tolist()
            assert (row[dg:] == -1).all()


def test_prune_completeness():
    # every candidate skipped before the R-th keep has an occluder among the keeps
    base = datagen.uniform_int(300, 8, seed=38)
    D = sqdist_matrix(base, base)
    p = 5
    order = sorted((D[p, q], q) for q in range(300) if q != p)[:100]
    ids = np.array([q for _, q in order], np.int32)
    dist = np.array([d for d, _ in order], np.float32)
    row, dg = oracle.prune(base, ids, dist, 12)
    kept = row[:dg].tolist()
    last = ids.tolist().index(kept[-1])
    for t in range(last + 1):
        q = int(ids[t])
        if q in kept:
            continue
        earlier = kept[: [i for i, k in enumerate(kept) if ids.tolist().index(k) < t][-1] + 1]
        assert any(D[q, r] < D[p, q] for r in earlier)
