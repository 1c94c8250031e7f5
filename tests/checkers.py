"""Independent checkers built from the paper's definitions and library routines.

None of these calls the oracle or the CUDA path.  They evaluate a definition
directly (Def. MRNG, Lemma 1's MSNET criterion, Eq. 1 precision, reachability
from the navigating node) or reduce to a numpy / scipy routine, so that the
oracle and the CUDA path are both checked against something other than
themselves.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order


def sqdist_matrix(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Exact squared l2 distances in float64 (exact on small integer data)."""
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    return ((a[:, None, :] - b[None, :, :]) ** 2).sum(-1)


def brute_knn(base: np.ndarray, queries: np.ndarray, k: int, exclude_self: bool = False):
    """k nearest by (squared distance, id) using np.lexsort; self excluded by id."""
    D = sqdist_matrix(queries, base)
    n = base.shape[0]
    ids = np.empty((len(queries), k), np.int64)
    dist = np.empty((len(queries), k), np.float64)
    col = np.arange(n)
    for i in range(len(queries)):
        keep = col != i if exclude_self else np.ones(n, bool)
        c, dd = col[keep], D[i][keep]
        order = np.lexsort((c, dd))[:k]
        ids[i], dist[i] = c[order], dd[order]
    return ids, dist


def edges_of(adj: np.ndarray, deg=None):
    out = []
    for p in range(adj.shape[0]):
        row = adj[p][: deg[p]] if deg is not None else adj[p][adj[p] >= 0]
        out.append([int(x) for x in row])
    return out


def reachable(adj: np.ndarray, deg: np.ndarray, root: int) -> np.ndarray:
    """Boolean mask of nodes reachable from root (scipy BFS)."""
    n = adj.shape[0]
    rows, cols = [], []
    for p in range(n):
        for q in adj[p][: deg[p]]:
            if q >= 0:
                rows.append(p)
                cols.append(int(q))
    g = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    order = breadth_first_order(g, root, directed=True, return_predecessors=False)
    mask = np.zeros(n, bool)
    mask[order] = True
    return mask


def key_before(d2_a: float, id_a: int, d2_b: float, id_b: int) -> bool:
    return d2_a < d2_b or (d2_a == d2_b and id_a < id_b)


def mrng_fixpoint_violations(base: np.ndarray, edges) -> list:
    """Def. MRNG as a fixpoint over a given edge set.

    p->q must be an edge  iff  no r with p->r an edge lies in the lune of pq.
    The lune is the intersection of the open balls B(p, |pq|) and B(q, |pq|);
    with the index tie rule, "r in B(p, |pq|)" reads "r precedes q in the
    (distance to p, id) order".  The definition's recursion only looks at
    points nearer to p, so exactly one edge set satisfies it for all pairs.
    Returns the list of violating (p, q) pairs."""
    D = sqdist_matrix(base, base)
    n = len(base)
    bad = []
    for p in range(n):
        E = set(edges[p])
        for q in range(n):
            if q == p:
                continue
            blocked = any(
                key_before(D[p, r], r, D[p, q], q) and D[q, r] < D[p, q] for r in E if r != q
            )
            if (q in E) == blocked:
                bad.append((p, q))
    return bad


def msnet_violations(base: np.ndarray, edges) -> list:
    """Lemma 1: G is an MSNET iff for every p != q some edge p->r has r in the
    open ball B(q, |pq|) (r = q allowed).  Returns violating pairs."""
    D = sqdist_matrix(base, base)
    n = len(base)
    bad = []
    for p in range(n):
        for q in range(n):
            if p != q and not any(D[r, q] < D[p, q] for r in edges[p]):
                bad.append((p, q))
    return bad


def occlusion_violations(base: np.ndarray, adj: np.ndarray, deg: np.ndarray, nodes=None) -> list:
    """MRNG property of each selected row: for kept r listed before p in v's row,
    |p - r|^2 >= |p - v|^2 (p is not in any earlier edge's lune)."""
    bad = []
    nodes = range(adj.shape[0]) if nodes is None else nodes
    for v in nodes:
        row = [int(x) for x in adj[v][: deg[v]]]
        X = base[row].astype(np.float64)
        dv = ((X - base[v].astype(np.float64)) ** 2).sum(1)
        for a in range(len(row)):
            for b in range(a):
                if ((X[a] - X[b]) ** 2).sum() < dv[a]:
                    bad.append((v, row[b], row[a]))
    return bad


def precision(ids: np.ndarray, gt: np.ndarray, k: int) -> float:
    """Eq. 1: |R' n R| / K averaged over queries."""
    hits = 0
    for a, b in zip(ids[:, :k], gt[:, :k]):
        hits += len(set(int(x) for x in a if x >= 0) & set(int(x) for x in b))
    return hits / float(len(ids) * k)


def read_golden(path: str):
    """Parse a golden text file into a list of (tag, [values]) records."""
    recs = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            recs.append((parts[0], parts[1:]))
    return recs
