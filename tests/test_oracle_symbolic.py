"""Pins of the oracle's symbolic factor count (oracle/symbolic.py).

The count is the byte floor of the local triangular solves (every entry of every L_i of
Algorithm 1 is read once per sweep).  It is checked against closed forms and against
the nonzeros of numerical Cholesky factors -- never against itself.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import algmortar as oa
from oracle import partition as op
from oracle import symbolic as osym


def spd_with_pattern(P, seed):
    """Random SPD matrix whose off-diagonal nonzeros are exactly those of P (generic
    values: no cancellation in the factor)."""
    P = sp.coo_matrix(P)
    rng = np.random.default_rng(seed)
    off = P.row != P.col
    r, c = P.row[off], P.col[off]
    keep = r < c
    v = -rng.uniform(0.5, 1.5, keep.sum())
    n = P.shape[0]
    M = sp.coo_matrix((np.concatenate([v, v]), (np.concatenate([r[keep], c[keep]]),
                                                np.concatenate([c[keep], r[keep]]))), shape=(n, n)).tocsr()
    d = np.asarray(abs(M).sum(axis=1)).ravel() + rng.uniform(0.5, 1.5, n)
    return (M + sp.diags(d)).tocsr()


def numeric_nnz(A, order=None):
    D = A.toarray()
    if order is not None:
        D = D[np.ix_(order, order)]
    L = np.linalg.cholesky(D)
    return int((np.abs(L) > 1e-13 * np.abs(L).max()).sum())


def grid2d(k):
    I = sp.identity(k)
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(k, k))
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_tridiagonal_has_no_fill(n):
    A = spd_with_pattern(sp.diags([1.0, 1.0, 1.0], [-1, 0, 1], shape=(n, n)), 1)
    assert osym.factor_nnz(A) == 2 * n - 1
    assert osym.factor_nnz(A, osym.fill_reducing_order(A)) == 2 * n - 1


@pytest.mark.parametrize("n", [1, 5, 23])
def test_dense_fills_the_triangle(n):
    A = spd_with_pattern(np.ones((n, n)), 2)
    for order in (None, np.random.default_rng(3).permutation(n)):
        assert osym.factor_nnz(A, order) == n * (n + 1) // 2


def test_arrow_hub_last_and_first():
    """Star graph: eliminating the hub last gives no fill (2n - 1); first, a full triangle."""
    n = 17
    P = sp.lil_matrix((n, n))
    P.setdiag(1.0)
    P[0, :] = 1.0
    P[:, 0] = 1.0
    A = spd_with_pattern(P, 4)
    hub_last = np.r_[np.arange(1, n), 0]
    assert osym.factor_nnz(A, hub_last) == 2 * n - 1
    assert osym.factor_nnz(A) == n * (n + 1) // 2
    assert osym.factor_nnz(A, osym.fill_reducing_order(A)) == 2 * n - 1


@pytest.mark.parametrize("k", [3, 5, 8, 11])
def test_grid_natural_order_band(k):
    """k x k five-point grid, natural order: the first grid row is a path (2 entries a
    row after the first), and every later row i fills its envelope i-k .. i."""
    A = grid2d(k)
    n = k * k
    assert osym.factor_nnz(A) == 1 + 2 * (k - 1) + (n - k) * (k + 1)


def test_random_tree_has_no_fill_under_minimum_degree():
    rng = np.random.default_rng(5)
    n = 60
    parent = [int(rng.integers(0, i)) for i in range(1, n)]
    P = sp.coo_matrix((np.ones(n - 1), (np.arange(1, n), parent)), shape=(n, n))
    A = spd_with_pattern(P + P.T + sp.identity(n), 6)
    assert osym.factor_nnz(A, osym.fill_reducing_order(A)) == 2 * n - 1


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_symbolic_equals_numerical_factor(seed):
    """Random sparse patterns: the symbolic count equals the nonzeros of the dense
    numerical Cholesky factor, under the natural, a random and the fill-reducing order."""
    rng = np.random.default_rng(seed)
    n = 45
    P = sp.random(n, n, density=0.06, random_state=seed)
    P = ((P + P.T) != 0).astype(float) + sp.identity(n)
    A = spd_with_pattern(P, seed)
    for order in (None, rng.permutation(n), osym.fill_reducing_order(A)):
        assert osym.factor_nnz(A, order) == numeric_nnz(A, order)


def test_fill_reducing_order_beats_natural_on_3d_grid():
    lnK = synth.gaussian_field((7, 6, 5), 2.0, 1.0, 12)
    A, _ = synth.tpfa_cartesian(np.exp(lnK))
    natural = osym.factor_nnz(A)
    mmd = osym.factor_nnz(A, osym.fill_reducing_order(A))
    assert mmd < natural
    assert mmd == numeric_nnz(A, osym.fill_reducing_order(A))


def test_local_factor_nnz_counts_every_subdomain():
    """sum_i nnz(L_i) over the local matrices A_i of Eq. (A_i) equals the nonzeros of
    their numerical factors under the same orders."""
    lnK = synth.gaussian_field((9, 8, 4), 2.0, 1.5, 13)
    A, _ = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1)
    part = op.partition(A, synth.even_part_sizes(A.shape[0], 5))
    pc = oa.setup(A, part)
    total = osym.local_factor_nnz(pc.A_loc)
    ref = sum(numeric_nnz(Ai, osym.fill_reducing_order(Ai)) for Ai in pc.A_loc)
    assert total == ref
