"""Inexact interface solve of Algorithm 2 -- oracle, TEST INFRASTRUCTURE ONLY.

Sec. 7 (the paper's solver settings): the interface system S eta = b_eta of Algorithm 2
("solve the interface system") is solved by an inner PCG with a block-Jacobi
preconditioner to a relative tolerance of 1e-2 instead of exactly.  cal_M^{-1} then
depends non-linearly on r, so the outer CG takes the flexible (Polak-Ribiere) beta
(`algmortar.pcg(..., flexible=True)`).

Readings taken where the paper is silent (its runs use the PETSc defaults of the
interface KSP):

* Blocks.  Interface I = (i, j), i < j, belongs to block floor(i / g): the interfaces
  owned by g consecutive subdomain ids, which recursive bisection keeps spatially
  together.  Interfaces are numbered lexicographically by (i, j), so every block is a
  contiguous range of interface ids.  Each block is solved exactly with the inverse of
  S restricted to it (symmetrised: the exact inverse is symmetric).
* Stop.  eta_0 = 0 and ||b - S eta_k||_2 <= rtol ||b||_2 on the recurrence residual,
  like the outer PCG; at most `max_it` products with S; a non-positive p . S p stops.
* Arithmetic.  `dtype` float64, or float32 for S, the block inverses (formed in FP64,
  rounded once), and every vector; dot products are accumulated in FP64 and alpha, beta
  are rounded to float32 where they scale a vector.  The stop test compares FP64 sums.

Pinned by tests/test_oracle_inexact.py: iterates equal to scipy's preconditioned CG, a
single block gives the exact solve in one step, the stop rule and its minimality, the
float32 mode against FP64, and the tight-tolerance limit equal to Algorithm 2's exact
interface solve.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from .algmortar import Preconditioner


def interface_blocks(pairs: np.ndarray, g: int) -> List[np.ndarray]:
    """Block-Jacobi blocks of the interface unknowns: I = (i, j) -> block i // g."""
    owner = np.asarray(pairs)[:, 0] // int(g)
    if owner.size and np.any(np.diff(owner) < 0):
        raise ValueError("interfaces must be numbered lexicographically by (i, j)")
    _, start = np.unique(owner, return_index=True)
    bounds = np.append(start, owner.size)
    return [np.arange(bounds[t], bounds[t + 1]) for t in range(len(start))]


def block_inverses(S: np.ndarray, blocks: List[np.ndarray], dtype=np.float64) -> List[np.ndarray]:
    """Symmetrised inverse of each diagonal block S[b, b] (FP64), rounded once to dtype."""
    out = []
    for b in blocks:
        X = np.linalg.inv(S[np.ix_(b, b)])
        out.append((0.5 * (X + X.T)).astype(dtype))
    return out


def _dot(u: np.ndarray, v: np.ndarray) -> float:
    return float(np.dot(u.astype(np.float64), v.astype(np.float64)))


def inner_pcg(S: np.ndarray, b: np.ndarray, blocks: List[np.ndarray], Binv: List[np.ndarray],
              rtol: float, max_it: int, dtype=np.float64):
    """PCG on S eta = b with the block-Jacobi preconditioner; returns (eta, iterations)
    with eta as float64 (the values of the dtype iterate)."""
    f = np.dtype(dtype).type
    Sf = np.asarray(S, dtype=dtype)
    bf = np.asarray(b, dtype=np.float64).astype(dtype)

    def prec(r):
        z = np.empty_like(r)
        for blk, Bi in zip(blocks, Binv):
            z[blk] = Bi @ r[blk]
        return z

    x = np.zeros_like(bf)
    bb = _dot(bf, bf)
    if bb == 0.0:
        return x.astype(np.float64), 0
    r = bf.copy()
    z = prec(r)
    p = z.copy()
    rz = _dot(r, z)
    tol2 = rtol * rtol * bb
    it = 0
    for it in range(1, max_it + 1):
        q = Sf @ p
        pq = _dot(p, q)
        if not np.isfinite(pq) or pq <= 0.0:
            return x.astype(np.float64), it
        alpha = rz / pq
        x = x + f(alpha) * p
        r = r - f(alpha) * q
        if _dot(r, r) <= tol2:
            return x.astype(np.float64), it
        z = prec(r)
        rz_new = _dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + f(beta) * p
    return x.astype(np.float64), it


@dataclasses.dataclass
class InexactInterface:
    """Block-Jacobi data of the inexact interface solve for one setup."""
    blocks: List[np.ndarray]
    Binv: List[np.ndarray]
    dtype: type
    iterations: List[int] = dataclasses.field(default_factory=list)


def inexact_setup(pc: Preconditioner, g: int, dtype=np.float64) -> InexactInterface:
    blocks = interface_blocks(pc.sk.pairs, g)
    return InexactInterface(blocks, block_inverses(pc.S, blocks, dtype), dtype)


def apply_inexact(pc: Preconditioner, ii: InexactInterface, r: np.ndarray, rtol: float = 1e-2,
                  max_it: int = 200) -> np.ndarray:
    """Algorithm 2 with the interface system solved by `inner_pcg` (original ordering);
    the inner iteration count is appended to ii.iterations."""
    sk = pc.sk
    f = np.asarray(r, dtype=np.float64)[sk.perm]
    pbar = np.empty_like(f)
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        pbar[a:b] = pc.lu[i].solve(f[a:b])
    rhs = -(pc.Z.T @ (pc.W @ (pc.M @ pbar)))
    eta, its = inner_pcg(pc.S, rhs, ii.blocks, ii.Binv, rtol, max_it, ii.dtype)
    ii.iterations.append(its)
    p = pbar.copy()
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        if pc.I_loc[i].size:
            p[a:b] += pc.Phat[i] @ eta[pc.I_loc[i]]
    return p[sk.iperm]
