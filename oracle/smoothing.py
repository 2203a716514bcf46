"""Block-Jacobi pre- and post-smoothing around the AlgMortar correction -- oracle.

Test infrastructure only (like the rest of `oracle/`): plain FP64 numpy/scipy, slow and
direct, never imported by the product package.

Sec. 5.4 (smoothing steps): AlgMortar leaves residuals only on the partition interface;
the paper reduces them with block-Jacobi smoothing applied the same number of times
before and after the AlgMortar correction, composed multiplicatively (Sec. 6: PETSc's
block Jacobi combined with the shell preconditioner; Sec. 7: 15 + 15 steps).  For an
input residual r the composite preconditioner computes

    x = 0
    nu times:  x <- x + B^{-1} (r - A x)            (pre-smoothing)
               x <- x + M_AM^{-1} (r - A x)         (AlgMortar, Algorithm 2)
    nu times:  x <- x + B^{-1} (r - A x)            (post-smoothing)

with B = blockdiag(A_bb) over the smoother blocks b.  Readings where the paper is
silent: the blocks are unions of whole AlgMortar subdomains (`group` consecutive
subdomain labels per block; the paper uses fewer, larger blocks than subdomains), and
each block is solved exactly (a sparse LU here) where PETSc's default sub-solver is
ILU(0).  nu = 0 gives Algorithm 2 unchanged.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import algmortar as oa


@dataclasses.dataclass
class BlockJacobi:
    blocks: List[np.ndarray]      # original-order indices of each block
    lu: list                      # SuperLU of A restricted to each block


def block_jacobi_setup(A: sp.spmatrix, part: np.ndarray, group: int = 1) -> BlockJacobi:
    """Blocks b = { k : part[k] // group == b }, each with the exact factor of A_bb."""
    A = sp.csr_matrix(A)
    lab = np.asarray(part) // int(group)
    blocks, lu = [], []
    for b in range(int(lab.max()) + 1):
        idx = np.flatnonzero(lab == b)
        if idx.size == 0:
            continue
        blocks.append(idx)
        lu.append(spla.splu(sp.csc_matrix(A[idx][:, idx])))
    return BlockJacobi(blocks, lu)


def block_jacobi_solve(bj: BlockJacobi, s: np.ndarray) -> np.ndarray:
    """y = B^{-1} s, block by block (original ordering)."""
    y = np.zeros_like(s)
    for idx, f in zip(bj.blocks, bj.lu):
        y[idx] = f.solve(s[idx])
    return y


def smoothed_apply(A: sp.spmatrix, pc: oa.Preconditioner, bj: BlockJacobi, r: np.ndarray,
                   nu: int) -> np.ndarray:
    """The composite preconditioner above, original ordering in and out."""
    A = sp.csr_matrix(A)
    r = np.asarray(r, dtype=np.float64)
    x = np.zeros_like(r)
    for _ in range(nu):
        x = x + block_jacobi_solve(bj, r - A @ x)
    x = x + oa.apply(pc, r - A @ x)
    for _ in range(nu):
        x = x + block_jacobi_solve(bj, r - A @ x)
    return x
