"""Pins of the smoothing oracle (Sec. 5.4: block-Jacobi pre/post smoothing composed with
the AlgMortar correction).  Each check compares against something other than the loop
itself: closed-form error propagation built from dense inverses, a direct solve, the
unsmoothed Algorithm 2, symmetry and the spectrum of the preconditioned operator."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import algmortar as oa
from oracle import partition as op
from oracle import smoothing as osm


def problem(shape=(8, 6, 1), sigma=1.0, seed=11, m=4):
    lnK = synth.gaussian_field(shape, 2.0, sigma, seed)
    A, f = synth.tpfa_cartesian(np.exp(lnK), bc_axis=0)
    part = op.partition(A, synth.even_part_sizes(A.shape[0], m))
    return sp.csr_matrix(A), f, part


@pytest.fixture(scope="module")
def p3():
    A, f, part = problem(shape=(6, 5, 4), sigma=1.5, seed=5, m=6)
    return A, f, part, oa.setup(A, part)


def dense_precond(fun, n):
    return np.column_stack([fun(e) for e in np.eye(n)])


def test_nu0_is_algorithm2(p3):
    A, f, part, pc = p3
    bj = osm.block_jacobi_setup(A, part)
    r = np.random.default_rng(1).standard_normal(A.shape[0])
    np.testing.assert_array_equal(osm.smoothed_apply(A, pc, bj, r, 0), oa.apply(pc, r))


def test_block_solve_is_block_diagonal_inverse(p3):
    """B^{-1} s against the dense inverse of blockdiag(A_bb), blocks of 2 subdomains."""
    A, f, part, pc = p3
    bj = osm.block_jacobi_setup(A, part, group=2)
    Ad = A.toarray()
    Bd = np.zeros_like(Ad)
    lab = part // 2
    for b in np.unique(lab):
        idx = np.flatnonzero(lab == b)
        Bd[np.ix_(idx, idx)] = Ad[np.ix_(idx, idx)]
    s = np.random.default_rng(2).standard_normal(A.shape[0])
    y = osm.block_jacobi_solve(bj, s)
    assert np.linalg.norm(y - np.linalg.solve(Bd, s)) <= 1e-12 * np.linalg.norm(y)


@pytest.mark.parametrize("nu,group", [(1, 1), (2, 1), (1, 3)])
def test_error_propagation_closed_form(p3, nu, group):
    """I - M_s^{-1} A = (I - B^{-1} A)^nu (I - M^{-1} A) (I - B^{-1} A)^nu, with B^{-1}
    from dense inverses of the blocks and M^{-1} from the dense reduced operator of
    Eq. (eq-m-reduced-p)."""
    A, f, part, pc = p3
    n = A.shape[0]
    Ad = A.toarray()
    lab = part // group
    Binv = np.zeros_like(Ad)
    for b in np.unique(lab):
        idx = np.flatnonzero(lab == b)
        Binv[np.ix_(idx, idx)] = np.linalg.inv(Ad[np.ix_(idx, idx)])
    Minv = dense_precond(lambda e: oa.apply_dense(pc, e), n)
    I = np.eye(n)
    Es = np.linalg.matrix_power(I - Binv @ Ad, nu)
    E = Es @ (I - Minv @ Ad) @ Es
    bj = osm.block_jacobi_setup(A, part, group=group)
    Ms = dense_precond(lambda e: osm.smoothed_apply(A, pc, bj, e, nu), n)
    assert np.abs((I - Ms @ Ad) - E).max() <= 1e-9


@pytest.mark.parametrize("nu", [1, 2])
def test_symmetric_and_spectrum_in_unit_interval(p3, nu):
    """Equal pre/post counts keep M_s^{-1} symmetric; with a convergent smoother the
    eigenvalues of M_s^{-1} A lie in (0, 1] and the smallest one does not drop below the
    unsmoothed one."""
    A, f, part, pc = p3
    n = A.shape[0]
    bj = osm.block_jacobi_setup(A, part)
    Ms = dense_precond(lambda e: osm.smoothed_apply(A, pc, bj, e, nu), n)
    assert np.abs(Ms - Ms.T).max() <= 1e-12 * np.abs(Ms).max()
    Ad = A.toarray()
    L = np.linalg.cholesky(Ad)
    lam = np.linalg.eigvalsh(L.T @ Ms @ L)
    M0 = dense_precond(lambda e: oa.apply(pc, e), n)
    lam0 = np.linalg.eigvalsh(L.T @ M0 @ L)
    assert lam.min() > 0 and lam.max() <= 1 + 1e-10
    assert lam.min() >= lam0.min() - 1e-12


def test_single_block_is_exact(p3):
    """One smoother block covering the whole domain: B = A, so one pre-smoothing step
    solves the system and the result is A^{-1} r."""
    A, f, part, pc = p3
    bj = osm.block_jacobi_setup(A, part, group=int(part.max()) + 1)
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    x = osm.smoothed_apply(A, pc, bj, r, 1)
    xs = spla.spsolve(sp.csc_matrix(A), r)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_smoothing_reduces_pcg_iterations():
    """Sec. 5.4's purpose on a 3D problem: nu = 1 takes fewer PCG iterations than nu = 0."""
    A, f, part = problem(shape=(12, 10, 8), sigma=2.0, seed=7, m=8)
    pc = oa.setup(A, part)
    bj = osm.block_jacobi_setup(A, part)
    it0 = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-8).iterations
    it1 = oa.pcg(A, f, lambda v: osm.smoothed_apply(A, pc, bj, v, 1), 1e-8).iterations
    assert it1 < it0
