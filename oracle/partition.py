"""Deterministic graph partition of the adjacency graph G(A) (Sec. 3.1) -- oracle.

The paper partitions G(A) = (Omega, E), (k, l) in E iff k != l and a_kl != 0, with
METIS/ParMETIS (Sec. 3.1, Sec. 6).  METIS is not available and is not deterministic
across versions, so both implementations here follow one written rule instead
(recursive BFS bisection with George-Liu pseudo-peripheral start nodes):

* `split(S, t[lo:hi])` assigns the node set S (sorted by index) to the parts lo..hi-1
  whose target sizes t sum to |S|.  With k = hi - lo parts: if k == 1 every node of S
  goes to part lo; otherwise k1 = k // 2, n1 = t[lo] + ... + t[lo+k1-1], the nodes of S
  are put in BFS order (below), the first n1 go to parts lo..lo+k1-1 and the rest to
  lo+k1..hi-1, each half recursively.
* BFS order of S: breadth-first search of the subgraph induced by S, visiting each
  node's neighbours in ascending index, started at the pseudo-peripheral node of the
  component of min(S); afterwards, while nodes of S are unvisited, a fresh BFS starts
  from the smallest unvisited node (no pseudo-peripheral search there).
* Pseudo-peripheral node (George & Liu 1979): v = min(S); repeat {BFS levels from v;
  among the nodes of the last level take u of minimum degree in the induced subgraph,
  ties to the smaller index; if ecc(u) > ecc(v) set v = u, else stop}; return v.

Breadth-first search itself is taken from scipy.sparse.csgraph (a library primitive);
test_oracle_partition pins it against a plain-Python queue BFS.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse import csgraph


def adjacency(A: sp.spmatrix) -> sp.csr_matrix:
    """Pattern of G(A): off-diagonal nonzeros of A (Sec. 3.1), sorted CSR, values 1."""
    A = sp.csr_matrix(A, copy=True)
    A.eliminate_zeros()
    G = A.tocoo()
    keep = G.row != G.col
    G = sp.csr_matrix((np.ones(int(keep.sum())), (G.row[keep], G.col[keep])), shape=A.shape)
    G.sort_indices()
    return G


def _dist(sub: sp.csr_matrix, start: int) -> np.ndarray:
    d = csgraph.shortest_path(sub, method="D", unweighted=True, directed=True, indices=start)
    return d


def pseudo_peripheral(sub: sp.csr_matrix) -> int:
    """George-Liu pseudo-peripheral node of the component of local node 0."""
    deg = np.diff(sub.indptr)
    v = 0
    d = _dist(sub, v)
    ecc = int(np.max(d[np.isfinite(d)]))
    while True:
        last = np.flatnonzero(d == ecc)
        u = int(last[np.lexsort((last, deg[last]))[0]])
        du = _dist(sub, u)
        ecc_u = int(np.max(du[np.isfinite(du)]))
        if ecc_u > ecc:
            v, d, ecc = u, du, ecc_u
        else:
            return v


def bfs_order(sub: sp.csr_matrix) -> np.ndarray:
    """BFS order (local indices) of all nodes of the induced subgraph `sub`."""
    n = sub.shape[0]
    seen = np.zeros(n, dtype=bool)
    parts = []
    start = pseudo_peripheral(sub)
    while True:
        order = csgraph.breadth_first_order(sub, start, directed=True,
                                            return_predecessors=False)
        seen[order] = True
        parts.append(order)
        rest = np.flatnonzero(~seen)
        if rest.size == 0:
            break
        start = int(rest[0])
    out = np.concatenate(parts).astype(np.int64)
    assert out.size == n
    return out


def partition(A: sp.spmatrix, sizes) -> np.ndarray:
    """Labels part[k] in [0, m) with |{k: part[k] == i}| == sizes[i] (Sec. 3.1)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    G = adjacency(A)
    n = G.shape[0]
    if sizes.sum() != n or (sizes <= 0).any():
        raise ValueError("part sizes must be positive and sum to N")
    part = np.empty(n, dtype=np.int32)
    stack = [(np.arange(n, dtype=np.int64), 0, len(sizes))]
    while stack:
        S, lo, hi = stack.pop()
        k = hi - lo
        if k == 1:
            part[S] = lo
            continue
        k1 = k // 2
        n1 = int(sizes[lo:lo + k1].sum())
        sub = G[S][:, S].tocsr()
        sub.sort_indices()
        order = bfs_order(sub)
        first = np.sort(S[order[:n1]])
        second = np.sort(S[order[n1:]])
        stack.append((second, lo + k1, hi))
        stack.append((first, lo, lo + k1))
    return part


def bfs_plain(indptr, indices, start, allowed=None):
    """Plain-Python FIFO BFS (neighbours in stored order); used only to pin csgraph."""
    n = len(indptr) - 1
    seen = [False] * n
    seen[start] = True
    q = [start]
    h = 0
    while h < len(q):
        u = q[h]
        h += 1
        for t in range(indptr[u], indptr[u + 1]):
            v = int(indices[t])
            if not seen[v] and (allowed is None or allowed[v]):
                seen[v] = True
                q.append(v)
    return q
