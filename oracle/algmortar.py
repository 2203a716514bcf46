"""AlgMortar preconditioner and PCG in plain FP64 numpy/scipy -- oracle.

Follows the paper's construction step by step, in its notation (the system is taken in
the permuted ordering after Sec. 3.1):

* E_ij, E_i, E                        Sec. 3.1, Eq. (E)
* C_ij, R, W, L, U, M, B_ij, B_i, B    Sec. 3.2, Eqs. (incidence-matrix), (global-W),
                                       (L-operator), (U-operator), (avg-operator),
                                       (Bij-matrix-form), (Bij-contrib), (def-B)
* D_ij, A_i, A_hat                     Sec. 3.3, Eqs. (Dij-def), (A_i)
* p_bar_i, MBFs p_hat_i^(m)            Sec. 3.4, Eqs. (def-pbar-local), (def-phat-local)
* interface problem                    Eqs. (interface-problem-alg-0), (interface-problem-alg)
* reduced preconditioner  cal_M        Cor. cor-schur-p, Eq. (eq-m-reduced-p)
* Algorithms 1 (setup) and 2 (apply)   Sec. 5.3
* interface space Lambda               Sec. 5.5: one piecewise-constant psi per E_ij
* PCG with x0 = 0 and a Euclidean relative-residual stop (Sec. 7)

Local factorisations use scipy's SuperLU (`splu`); dense factorisations use numpy's
LAPACK.  No blocking, fusion or reordering beyond what the paper states.

Reading taken where the paper is silent: unknowns are permuted stably by (part,
original index); interfaces (i, j), i < j, are numbered lexicographically; an edge of
E_ij is written (k, l) with k in Omega_i, l in Omega_j, i < j.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclasses.dataclass
class Skeleton:
    """Algebraic skeleton of a partition (Sec. 3.1-3.2), all in the permuted ordering."""

    perm: np.ndarray        # perm[new] = old
    iperm: np.ndarray       # iperm[old] = new
    offsets: np.ndarray     # Omega_i = [offsets[i], offsets[i+1])
    A: sp.csr_matrix        # permuted A = P A P^T (Eq. linear-system-perm)
    ek: np.ndarray          # edge e = (k, l): k in Omega_i
    el: np.ndarray          #                  l in Omega_j, i < j
    ea: np.ndarray          # a_kl
    eI: np.ndarray          # interface id of the edge (column of Z)
    pairs: np.ndarray       # pairs[I] = (i, j)

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def m(self):
        return len(self.offsets) - 1

    @property
    def nE(self):
        return len(self.ek)

    @property
    def nLam(self):
        return len(self.pairs)


def skeleton(A: sp.spmatrix, part: np.ndarray) -> Skeleton:
    """Permutation (Eq. linear-system-perm) and interface edge sets E_ij (Eq. E)."""
    A = sp.csr_matrix(A)
    part = np.asarray(part, dtype=np.int64)
    n = A.shape[0]
    m = int(part.max()) + 1
    perm = np.lexsort((np.arange(n), part))          # stable by (part, index)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    counts = np.bincount(part, minlength=m)
    if (counts == 0).any():
        raise ValueError("empty subdomain")
    offsets = np.concatenate([[0], np.cumsum(counts)])
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    Ap.eliminate_zeros()
    pp = part[perm]                                   # part of each permuted index
    coo = Ap.tocoo()
    sel = pp[coo.row] < pp[coo.col]                   # k in Omega_i, l in Omega_j, i < j
    ek, el, ea = coo.row[sel], coo.col[sel], coo.data[sel]
    pi, pj = pp[ek], pp[el]
    key = pi * m + pj
    ukeys, eI = np.unique(key, return_inverse=True)   # lexicographic (i, j)
    pairs = np.stack([ukeys // m, ukeys % m], axis=1)
    order = np.lexsort((el, ek, eI))                   # group edges by interface
    return Skeleton(perm, iperm, offsets, Ap, ek[order], el[order], ea[order],
                    eI[order].astype(np.int64), pairs)


def part_of(sk: Skeleton) -> np.ndarray:
    return np.repeat(np.arange(sk.m), np.diff(sk.offsets))


# ------------------------------------------------------------------ Sec. 3.2 operators

def operators(sk: Skeleton, mortar: str = "piecewise_constant"):
    """Sparse W, L, U, M, B, Z of Sec. 3.2 / 5.5 over the edge set E.

    W = diag(a_kl) (Eq. global-W); L p picks p at the endpoint in the lower-indexed
    subdomain (Eq. L-operator), U at the higher one (Eq. U-operator); M = (L + U) / 2
    (Eq. avg-operator); B is assembled entry by entry from Eq. (Bij-contrib):
    (B mu)_k = 2 sum_{l:(k,l) in E} a_kl mu(k,l) for each endpoint k of an edge.
    Z: columns spanning Lambda -- one indicator per interface E_ij (Sec. 5.5), or the
    identity of R^E when mortar == "edge" (Lambda = R^E, Eq. local-system-lm remark).
    """
    n, nE = sk.n, sk.nE
    e = np.arange(nE)
    W = sp.diags(sk.ea)
    L = sp.csr_matrix((np.ones(nE), (e, sk.ek)), shape=(nE, n))
    U = sp.csr_matrix((np.ones(nE), (e, sk.el)), shape=(nE, n))
    M = 0.5 * (L + U)
    B = sp.csr_matrix((np.concatenate([2.0 * sk.ea, 2.0 * sk.ea]),
                       (np.concatenate([sk.ek, sk.el]), np.concatenate([e, e]))),
                      shape=(n, nE))
    if mortar == "edge":
        Z = sp.identity(nE, format="csr")
    else:
        Z = sp.csr_matrix((np.ones(nE), (e, sk.eI)), shape=(nE, sk.nLam))
    return W, L, U, M, B, Z


def local_matrices(sk: Skeleton) -> List[sp.csc_matrix]:
    """A_i = A_ii - sum_{j~i} D_ij with D_ij = diag(A_ij 1)  (Eqs. Dij-def, A_i)."""
    out = []
    A = sk.A
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        rows = A[a:b]
        Aii = rows[:, a:b]
        rowsum_all = np.asarray(rows.sum(axis=1)).ravel()
        rowsum_in = np.asarray(Aii.sum(axis=1)).ravel()
        D = rowsum_all - rowsum_in                  # sum_j (A_ij 1)_k over j != i
        out.append(sp.csc_matrix(Aii - sp.diags(D)))
    return out


# ------------------------------------------------------------- Algorithms 1 and 2

@dataclasses.dataclass
class Preconditioner:
    sk: Skeleton
    mortar: str
    W: sp.spmatrix
    M: sp.spmatrix
    B: sp.spmatrix
    Z: sp.spmatrix
    A_loc: list
    lu: list
    I_loc: list            # I_i: interface basis indices active on Omega_i
    Phat: list             # Phat[i]: N_i x |I_i| MBFs on Omega_i (Eq. def-phat-local)
    S: np.ndarray          # interface matrix tested with the basis of Lambda
    S_chol: np.ndarray     # lower Cholesky factor of S


def setup(A: sp.spmatrix, part: np.ndarray, mortar: str = "piecewise_constant") -> Preconditioner:
    """Algorithm 1 (AlgMortarSetup).

    Partition given; permute; for each i: A_i (diagonally modified A_ii), its factor,
    and MBFs p_hat^(m) solving A_i p_hat = -B_i psi_m for m in I_i; then the interface
    matrix from Eq. (interface-problem-alg-0) tested with the basis psi of Lambda:
        S = Z^T W (M P_hat - Z),   P_hat = [p_hat(psi_1) ... p_hat(psi_NLam)],
    which equals -Z^T (W M A_hat^{-1} B + W) Z, the Schur complement S_eta of
    Cor. cor-schur-eta, and must be SPD.
    """
    sk = skeleton(A, part)
    W, L, U, M, B, Z = operators(sk, mortar)
    A_loc = local_matrices(sk)
    lu = [spla.splu(Ai) for Ai in A_loc]
    BZ = sp.csr_matrix(B @ Z)
    WM = sp.csc_matrix(Z.T @ W @ M)                 # Z^T W M : Lambda-coeffs x N
    nL = Z.shape[1]
    S = np.asarray((Z.T @ W @ Z).todense()) * -1.0   # - Z^T W Z
    I_loc, Phat = [], []
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        Bi = BZ[a:b]                                # B_i psi_m for all m
        cols = np.unique(Bi.indices)               # I_i
        rhs = -np.asarray(Bi[:, cols].todense())
        Ph = lu[i].solve(rhs) if cols.size else np.zeros((b - a, 0))
        I_loc.append(cols)
        Phat.append(Ph)
        if cols.size:
            S[:, cols] += np.asarray((WM[:, a:b] @ Ph))
    S_chol = np.linalg.cholesky(S)                  # raises if S is not SPD
    return Preconditioner(sk, mortar, W, M, B, Z, A_loc, lu, I_loc, Phat, S, S_chol)


def apply(pc: Preconditioner, r: np.ndarray) -> np.ndarray:
    """Algorithm 2 (AlgMortarApply): z = cal_M^{-1} r, r and z in ORIGINAL ordering.

    p_bar_i = A_i^{-1} f_i; interface RHS b = -Z^T W M p_bar (Eq. interface-problem-alg-0
    tested with psi); S eta = b; p_i = p_bar_i + sum_{m in I_i} eta_m p_hat_i^(m).
    """
    sk = pc.sk
    f = np.asarray(r, dtype=np.float64)[sk.perm]
    pbar = np.empty_like(f)
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        pbar[a:b] = pc.lu[i].solve(f[a:b])
    rhs = -(pc.Z.T @ (pc.W @ (pc.M @ pbar)))
    y = sla.solve_triangular(pc.S_chol, rhs, lower=True)
    eta = sla.solve_triangular(pc.S_chol.T, y, lower=False)
    p = pbar.copy()
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        if pc.I_loc[i].size:
            p[a:b] += pc.Phat[i] @ eta[pc.I_loc[i]]
    return p[sk.iperm]


def apply_parts(pc: Preconditioner, r: np.ndarray):
    """Intermediate quantities of Algorithm 2 in the permuted ordering
    (p_bar, interface RHS b, eta, z) -- for stage-by-stage comparisons."""
    sk = pc.sk
    f = np.asarray(r, dtype=np.float64)[sk.perm]
    pbar = np.empty_like(f)
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        pbar[a:b] = pc.lu[i].solve(f[a:b])
    rhs = -(pc.Z.T @ (pc.W @ (pc.M @ pbar)))
    eta = sla.cho_solve((pc.S_chol, True), rhs)
    p = pbar.copy()
    for i in range(sk.m):
        a, b = sk.offsets[i], sk.offsets[i + 1]
        if pc.I_loc[i].size:
            p[a:b] += pc.Phat[i] @ eta[pc.I_loc[i]]
    return pbar, rhs, eta, p


# ------------------------------------------------------------ dense reduced route

def dense_reduced(pc: Preconditioner) -> np.ndarray:
    """cal_M = A_hat + 4 M^T W Z (Z^T W Z)^{-1} Z^T W M (Eq. eq-m-reduced-p), permuted
    ordering, dense -- small N only."""
    Ahat = sp.block_diag(pc.A_loc).toarray()
    W = pc.W.toarray()
    M = pc.M.toarray()
    Z = pc.Z.toarray()
    ZWZ = Z.T @ W @ Z
    WM = W @ M
    return Ahat + 4.0 * (M.T @ W @ Z) @ np.linalg.solve(ZWZ, Z.T @ WM)


def apply_dense(pc: Preconditioner, r: np.ndarray) -> np.ndarray:
    """z = cal_M^{-1} r through the dense reduced matrix (original ordering)."""
    sk = pc.sk
    Mm = dense_reduced(pc)
    z = np.linalg.solve(Mm, np.asarray(r, dtype=np.float64)[sk.perm])
    return z[sk.iperm]


# ----------------------------------------------------------------------------- PCG

@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    rel_residual: float       # true ||b - A x|| / ||b||
    converged: bool
    history: list


def pcg_iterations(A: sp.spmatrix, b: np.ndarray, precond, tol: float = 1e-8, max_it: int = 10000,
                   flexible: bool = False):
    """Preconditioned CG (Hestenes-Stiefel), x0 = 0, stop when ||r_k||_2 <= tol ||b||_2
    (the Euclidean relative residual of Sec. 7), confirmed on the true residual
    b - A x; if the confirmation fails the iteration continues.  `precond(r)` returns
    z = M^{-1} r.  beta = rho_{k+1} / rho_k, or with `flexible` the Polak-Ribiere
    (rho_{k+1} - r_{k+1} . z_k) / rho_k, equal in exact arithmetic for a linear SPD
    preconditioner and robust to a preconditioner that varies between iterations (the
    inexact interface solve).  A generator: it yields after every product with A (so
    that a caller can spread one solve over several timed pieces) and returns the
    PCGResult.
    """
    A = sp.csr_matrix(A)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return PCGResult(x, 0, 0.0, True, [])
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    hist = [1.0]
    it = 0
    for it in range(1, max_it + 1):
        q = A @ p
        pq = float(p @ q)
        if not np.isfinite(pq) or pq <= 0.0:
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        rn = float(np.linalg.norm(r))
        hist.append(rn / bn)
        if rn <= tol * bn:
            true = float(np.linalg.norm(b - A @ x))
            if true <= tol * bn:
                return PCGResult(x, it, true / bn, True, hist)
        rz_mix = float(r @ z) if flexible else 0.0
        z = precond(r)
        rz_new = float(r @ z)
        beta = (rz_new - rz_mix) / rz
        rz = rz_new
        p = z + beta * p
        yield it
    true = float(np.linalg.norm(b - A @ x))
    return PCGResult(x, it, true / bn, False, hist)


def pcg(A: sp.spmatrix, b: np.ndarray, precond, tol: float = 1e-8, max_it: int = 10000,
        flexible: bool = False) -> PCGResult:
    """PCG of `pcg_iterations` run to its stop (`iterations` counts products with A)."""
    gen = pcg_iterations(A, b, precond, tol, max_it, flexible)
    while True:
        try:
            next(gen)
        except StopIteration as stop:
            return stop.value
