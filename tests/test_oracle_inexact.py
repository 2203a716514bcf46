"""Pins of the oracle's inexact interface solve (Sec. 7 solver settings) and of the
flexible outer PCG, each against something other than the oracle itself: scipy's
preconditioned CG, the exact dense solve, the stop rule, and the tight-tolerance limit."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import algmortar as oa
from oracle import inexact as oi
from oracle import partition as op


def spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T


def contiguous_blocks(n, sizes):
    b, out = 0, []
    for s in sizes:
        out.append(np.arange(b, b + s))
        b += s
    assert b == n
    return out


def test_blocks_by_hand():
    pairs = np.array([[0, 1], [0, 2], [1, 2], [2, 3], [3, 4], [4, 5]])
    blocks = oi.interface_blocks(pairs, 2)
    assert [b.tolist() for b in blocks] == [[0, 1, 2], [3, 4], [5]]
    assert [b.tolist() for b in oi.interface_blocks(pairs, 100)] == [[0, 1, 2, 3, 4, 5]]
    assert [b.tolist() for b in oi.interface_blocks(pairs, 1)] == [[0, 1], [2], [3], [4], [5]]
    with pytest.raises(ValueError):
        oi.interface_blocks(pairs[::-1], 2)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_iterates_equal_scipy_cg(k):
    n = 40
    S = spd(n, 1e3, 3)
    b = np.random.default_rng(4).standard_normal(n)
    blocks = contiguous_blocks(n, [5, 9, 6, 10, 10])
    Binv = oi.block_inverses(S, blocks)

    def prec(r):
        z = np.empty_like(r)
        for blk, Bi in zip(blocks, Binv):
            z[blk] = Bi @ r[blk]
        return z

    x, its = oi.inner_pcg(S, b, blocks, Binv, 0.0, k)
    assert its == k
    M = spla.LinearOperator((n, n), matvec=prec, dtype=np.float64)
    xs, _ = spla.cg(S, b, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k, M=M)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_single_block_is_exact_in_one_step():
    n = 30
    S = spd(n, 1e4, 7)
    b = np.random.default_rng(8).standard_normal(n)
    blocks = [np.arange(n)]
    x, its = oi.inner_pcg(S, b, blocks, oi.block_inverses(S, blocks), 1e-10, 50)
    assert its == 1
    ref = np.linalg.solve(S, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_diagonal_system_with_unit_blocks():
    d = np.geomspace(1.0, 1e6, 12)
    S = np.diag(d)
    b = np.arange(1.0, 13.0)
    blocks = [np.array([i]) for i in range(12)]
    x, its = oi.inner_pcg(S, b, blocks, oi.block_inverses(S, blocks), 1e-12, 5)
    assert its == 1
    assert np.allclose(x, b / d, rtol=1e-15, atol=0.0)


def test_stop_rule_and_minimality():
    n = 60
    S = spd(n, 1e5, 9)
    b = np.random.default_rng(10).standard_normal(n)
    blocks = contiguous_blocks(n, [12] * 5)
    Binv = oi.block_inverses(S, blocks)
    x, its = oi.inner_pcg(S, b, blocks, Binv, 1e-2, 500)
    assert its > 1
    assert np.linalg.norm(b - S @ x) <= 1e-2 * np.linalg.norm(b) * (1 + 1e-9)
    x1, its1 = oi.inner_pcg(S, b, blocks, Binv, 1e-2, its - 1)
    assert its1 == its - 1
    assert np.linalg.norm(b - S @ x1) > 1e-2 * np.linalg.norm(b)


def test_zero_rhs():
    S = spd(8, 10.0, 1)
    x, its = oi.inner_pcg(S, np.zeros(8), [np.arange(8)], oi.block_inverses(S, [np.arange(8)]), 1e-2, 9)
    assert its == 0 and not x.any()


def test_float32_mode_tracks_fp64():
    n = 80
    S = spd(n, 30.0, 12)
    b = np.random.default_rng(13).standard_normal(n)
    blocks = contiguous_blocks(n, [16] * 5)
    x64, i64 = oi.inner_pcg(S, b, blocks, oi.block_inverses(S, blocks), 1e-3, 500)
    x32, i32 = oi.inner_pcg(S, b, blocks, oi.block_inverses(S, blocks, np.float32), 1e-3, 500, np.float32)
    assert i32 == i64 and i64 > 5
    assert np.linalg.norm(x32 - x64) <= 1e-5 * np.linalg.norm(x64)
    assert np.linalg.norm(b - S @ x32) <= 1.01e-3 * np.linalg.norm(b)


def small_pc(shape=(12, 10, 3), m=8, seed=21):
    lnK = synth.gaussian_field(shape, 2.0, 1.5, seed)
    A, f = synth.tpfa_cartesian(np.exp(lnK), bc_axis=0)
    part = op.partition(A, synth.even_part_sizes(A.shape[0], m))
    return A, f, oa.setup(A, part)


def test_tight_tolerance_is_algorithm2():
    A, f, pc = small_pc()
    ii = oi.inexact_setup(pc, 2)
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    z = oi.apply_inexact(pc, ii, r, rtol=1e-14, max_it=500)
    ref = oa.apply(pc, r)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)
    assert ii.iterations[-1] > 1


def test_loose_interface_solve_meets_its_tolerance():
    A, f, pc = small_pc()
    ii = oi.inexact_setup(pc, 2)
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    _, rhs, eta_exact, _ = oa.apply_parts(pc, r)
    eta, its = oi.inner_pcg(pc.S, rhs, ii.blocks, ii.Binv, 1e-2, 500)
    assert np.linalg.norm(rhs - pc.S @ eta) <= 1e-2 * np.linalg.norm(rhs) * (1 + 1e-9)
    assert np.linalg.norm(eta - eta_exact) > 1e-8 * np.linalg.norm(eta_exact)


def test_flexible_beta_equals_standard_for_linear_preconditioner():
    A, f, pc = small_pc()
    std = oa.pcg(A, f, lambda r: oa.apply(pc, r), tol=1e-10)
    flx = oa.pcg(A, f, lambda r: oa.apply(pc, r), tol=1e-10, flexible=True)
    assert std.converged and flx.converged
    assert abs(std.iterations - flx.iterations) <= 1
    assert np.linalg.norm(std.x - flx.x) <= 1e-8 * np.linalg.norm(std.x)


def test_flexible_outer_with_inexact_interface_converges():
    A, f, pc = small_pc()
    exact = oa.pcg(A, f, lambda r: oa.apply(pc, r), tol=1e-8)
    ii = oi.inexact_setup(pc, 2, np.float32)
    res = oa.pcg(A, f, lambda r: oi.apply_inexact(pc, ii, r, rtol=1e-2), tol=1e-8, flexible=True)
    assert res.converged and res.rel_residual <= 1e-8
    assert res.iterations >= exact.iterations - 1
    assert min(ii.iterations) >= 1
