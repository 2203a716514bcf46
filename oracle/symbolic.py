"""Symbolic size of the local Cholesky factors -- oracle (TEST INFRASTRUCTURE ONLY).

Algorithm 1 (Sec. 5.3) factors every local matrix A_i = L_i L_i^T; the paper's
implementation does so with a sparse Cholesky under a fill-reducing (AMD) ordering
(Sec. 6).  The number of entries of L_i under such an ordering is the byte floor of
the per-iteration local solves (two triangular sweeps read every entry of every L_i
once).  This module counts it:

* ``fill_reducing_order``: a fill-reducing symmetric ordering of A_i, taken from
  SuperLU's multiple-minimum-degree ordering on the pattern of A_i + A_i^T (a library
  primitive used as one step);
* ``factor_row_counts``: the plain symbolic elimination under a given ordering --
  row i of L holds the diagonal and every j < i reached from a neighbour j0 < i of i by
  walking up the elimination tree (parent(j) = first row below j with l_ij != 0) until
  a node already met for row i; each step of a walk is one entry of L;
* ``local_factor_nnz``: sum over the subdomains of nnz(L_i), for the local matrices
  A_i of Eq. (A_i) built by ``oracle.algmortar.local_matrices``.

Pinned by tests/test_oracle_symbolic.py against closed forms (tridiagonal, dense,
arrow with the hub last or first, the banded 2D grid under the natural order) and
against the nonzero count of numerical dense Cholesky factors of random matrices with
the same pattern.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def fill_reducing_order(Ai: sp.spmatrix) -> np.ndarray:
    """order[k] = index of A_i's row eliminated k-th (multiple minimum degree on
    A_i + A_i^T, from SuperLU; diagonal pivots, so the column permutation is the
    symmetric elimination order)."""
    Ai = sp.csc_matrix(Ai, copy=True)
    Ai.eliminate_zeros()
    n = Ai.shape[0]
    if n == 1:
        return np.zeros(1, dtype=np.int64)
    lu = spla.splu(Ai, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    pos = np.asarray(lu.perm_c, dtype=np.int64)    # column j is eliminated at pos[j]
    order = np.empty(n, dtype=np.int64)
    order[pos] = np.arange(n)
    return order


def factor_row_counts(Ai: sp.spmatrix, order=None) -> np.ndarray:
    """Entries of each row of L (diagonal included) for A_i eliminated in `order`
    (default: natural).  Plain symbolic elimination by elimination-tree walks."""
    A = sp.csr_matrix(Ai, copy=True)
    A.eliminate_zeros()                             # the pattern is a_kl != 0 (Sec. 3.1)
    n = A.shape[0]
    if order is None:
        order = np.arange(n)
    order = np.asarray(order, dtype=np.int64)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    parent = np.full(n, -1, dtype=np.int64)
    mark = np.full(n, -1, dtype=np.int64)
    counts = np.ones(n, dtype=np.int64)            # the diagonal
    indptr, indices = A.indptr, A.indices
    for i in range(n):                              # i: elimination step
        old = order[i]
        mark[i] = i
        for t in range(indptr[old], indptr[old + 1]):
            j = pos[indices[t]]
            if j >= i:
                continue
            while mark[j] != i:                     # walk up the tree from j
                mark[j] = i
                counts[i] += 1                      # l_ij != 0
                if parent[j] < 0:
                    parent[j] = i
                    break
                j = parent[j]
    return counts


def factor_nnz(Ai: sp.spmatrix, order=None) -> int:
    return int(factor_row_counts(Ai, order).sum())


def local_factor_nnz(A_loc) -> int:
    """sum_i nnz(L_i) under the fill-reducing order of each A_i (Algorithm 1's factors)."""
    return int(sum(factor_nnz(Ai, fill_reducing_order(Ai)) for Ai in A_loc))
