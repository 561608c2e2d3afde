"""Independent pins for the oracle: trussness and related quantities computed
straight from their definitions (paper §II), by methods that share nothing
with the oracle's peel.

* ``brute_truss``: for every k, Cohen's k-truss peel run from the whole graph
  (remove any edge lying in fewer than k-2 triangles of what is left, until
  nothing changes); trussness(e) = the largest k whose peel keeps e.  Pure
  Python sets, for graphs of a few dozen vertices.
* ``sparse_truss``: the same definition with triangle counts taken from the
  sparse product A·A (scipy), for graphs with a few thousand edges.
* ``coreness``: repeated removal of a minimum-degree vertex.
* ``triangle_count``: trace(A^3) / 6 with dense numpy.
"""
from __future__ import annotations

import numpy as np


def canon_edges(n, src, dst):
    """Canonical undirected edge list written plainly with Python sets."""
    s = set()
    for a, b in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        if a != b:
            s.add((min(a, b), max(a, b)))
    e = sorted(s)
    return (np.array([x for x, _ in e], np.int32), np.array([y for _, y in e], np.int32))


def _cohen_peel(edges, k):
    H = set(edges)
    adj = {}
    for u, v in H:
        adj.setdefault(u, set()).add(v)
        adj.setdefault(v, set()).add(u)
    changed = True
    while changed:
        changed = False
        for (u, v) in sorted(H):
            if (u, v) not in H:
                continue
            s = len(adj[u] & adj[v])
            if s < k - 2:
                H.discard((u, v))
                adj[u].discard(v)
                adj[v].discard(u)
                changed = True
    return H


def brute_truss(eu, ev):
    edges = list(zip(np.asarray(eu).tolist(), np.asarray(ev).tolist()))
    tau = {e: 2 for e in edges}
    k = 3
    while True:
        H = _cohen_peel(edges, k)
        if not H:
            break
        for e in H:
            tau[e] = k
        k += 1
    return np.array([tau[e] for e in edges], np.int32)


def _pick(M, rows, cols):
    """Entries M[rows[i], cols[i]] of a scipy sparse matrix as a flat array."""
    out = M[rows, cols]
    if hasattr(out, "toarray"):
        out = out.toarray()
    return np.asarray(out).ravel()


def sparse_truss(n, eu, ev):
    import scipy.sparse as sp

    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    m = eu.shape[0]
    tau = np.full(m, 2, np.int32)
    k = 3
    while True:
        alive = np.ones(m, bool)
        while True:
            idx = np.nonzero(alive)[0]
            A = sp.coo_matrix((np.ones(2 * idx.size), (np.concatenate([eu[idx], ev[idx]]),
                                                      np.concatenate([ev[idx], eu[idx]]))),
                              shape=(n, n)).tocsr()
            A2 = (A @ A).tocsr()
            s = _pick(A2, eu[idx], ev[idx])
            drop = idx[s < k - 2]
            if drop.size == 0:
                break
            alive[drop] = False
        if not alive.any():
            break
        tau[alive] = k
        k += 1
    return tau


def coreness(n, eu, ev):
    nbr = [set() for _ in range(n)]
    for u, v in zip(np.asarray(eu).tolist(), np.asarray(ev).tolist()):
        nbr[u].add(v)
        nbr[v].add(u)
    deg = [len(x) for x in nbr]
    # lazy min-heap of (current degree, vertex)
    import heapq
    heap = [(d, i) for i, d in enumerate(deg)]
    heapq.heapify(heap)
    alive = [True] * n
    core = [0] * n
    cur = 0
    while heap:
        d, v = heapq.heappop(heap)
        if not alive[v] or d != deg[v]:
            continue
        cur = max(cur, d)
        core[v] = cur
        alive[v] = False
        for w in nbr[v]:
            if alive[w]:
                deg[w] -= 1
                heapq.heappush(heap, (deg[w], w))
    return np.array(core, np.int32)


def triangle_count(n, eu, ev):
    # float64 products are exact here (entries stay far below 2^53)
    A = np.zeros((n, n), np.float64)
    A[eu, ev] = 1
    A[ev, eu] = 1
    return int(round(np.trace(A @ A @ A))) // 6


def support_dense(n, eu, ev):
    A = np.zeros((n, n), np.float64)
    A[eu, ev] = 1
    A[ev, eu] = 1
    return np.rint((A @ A)[eu, ev]).astype(np.int32)
