"""Inexact interface solve (Sec. 7 solver settings: block-Jacobi PCG on S_eta to a
relative tolerance, flexible outer CG) on the GPU against the oracle's inexact solve on the
same seeded inputs: the interface right-hand side element-wise, the inner stop rule in
FP64 against the oracle's S_eta, the oracle's FP32 inner PCG iterate, the prolongation of
the GPU's eta, and the outer PCG."""
import numpy as np
import pytest
import torch

import synth
from oracle import algmortar as oa
from oracle import inexact as oi
from oracle import partition as op

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    return max(float(np.linalg.norm(d)) / max(float(np.linalg.norm(b)), 1e-300),
               float(d.max(initial=0.0)) / max(float(np.abs(b).max(initial=0.0)), 1e-300))


def to_orig(v, perm):
    """A vector in a permuted ordering (perm[new] = old) in the original ordering."""
    out = np.empty_like(v)
    out[perm] = v
    return out


def problem(shape=(21, 17, 13), m=24, seed=31, sigma=2.0):
    lnK = synth.gaussian_field(shape, 3.0, sigma, seed)
    A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=1)
    sizes = synth.uneven_part_sizes(A.shape[0], m, 100, 600, seed)
    return A, f, sizes


@pytest.fixture(scope="module")
def case():
    A, f, sizes = problem()
    part = op.partition(A, sizes)
    return A, f, sizes, part, oa.setup(A, part)


def AM(A, sizes, **kw):
    from paper_2607_22905_b300.solver import AlgMortar
    return AlgMortar(A, len(sizes), part_sizes=sizes, interface_solve="inexact", **kw)


@pytest.mark.parametrize("g", [1, 2, 4])
def test_interface_solve_against_oracle(case, g):
    A, f, sizes, part, pc = case
    am = AM(A, sizes, iface_block_parts=g)
    info = am.get_info()
    assert info["interface_solve"] == 1 and info["iface_cluster"] >= 1
    assert info["iface_blocks"] == len(oi.interface_blocks(pc.sk.pairs, g))
    rng = np.random.default_rng(100 + g)
    for _ in range(2):
        r = rng.standard_normal(A.shape[0])
        pbar, beta, eta, z = (t.cpu().numpy() for t in am.apply_stages(r))
        pbar_o, rhs_o, eta_exact, _ = oa.apply_parts(pc, r)
        perm = am.permutation()                  # internal -> original
        assert rel(to_orig(pbar, perm), to_orig(pbar_o, pc.sk.perm)) <= 1e-10
        assert rel(beta, rhs_o) <= 1e-10
        its = am.get_info()["iface_last_iterations"]
        assert its >= 1
        # the inner stop rule, in FP64 against the oracle's S_eta (FP32 storage of S adds
        # rounding of order kappa(S) * 6e-8 to the true residual)
        res = np.linalg.norm(rhs_o - pc.S @ eta) / np.linalg.norm(rhs_o)
        assert res <= 1e-2 * 1.05
        # the oracle's FP32 inner PCG on the same right-hand side and blocks
        ii = oi.inexact_setup(pc, g, np.float32)
        eta_o, its_o = oi.inner_pcg(pc.S, rhs_o, ii.blocks, ii.Binv, 1e-2, 200, np.float32)
        assert abs(its - its_o) <= 1
        if its == its_o:
            assert rel(eta, eta_o) <= 2e-3
        # prolongation of the GPU's eta: z = pbar + sum_m eta_m p_hat^(m)
        zz = pbar_o.copy()
        for i in range(pc.sk.m):
            a, b = pc.sk.offsets[i], pc.sk.offsets[i + 1]
            if pc.I_loc[i].size:
                zz[a:b] += pc.Phat[i] @ eta[pc.I_loc[i]]
        assert rel(to_orig(z, perm), to_orig(zz, pc.sk.perm)) <= 1e-10


def test_one_block_gives_the_exact_solve(case):
    """g >= m: a single block holds every interface when n_lambda <= 128, so the inner PCG
    converges in one step to the block inverse's solution."""
    A, f, sizes = problem(shape=(12, 10, 6), m=6, seed=5)
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    assert pc.sk.nLam <= 128
    am = AM(A, sizes, iface_block_parts=1000)
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    _, beta, eta, _ = (t.cpu().numpy() for t in am.apply_stages(r))
    _, rhs_o, eta_exact, _ = oa.apply_parts(pc, r)
    assert am.get_info()["iface_last_iterations"] == 1
    assert rel(eta, eta_exact) <= 1e-5


def test_outer_flexible_pcg(case):
    A, f, sizes, part, pc = case
    am = AM(A, sizes, iface_block_parts=2)
    x, st = am.solve(f, tol=1e-8, history=400)
    x = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(f - A @ x) <= 1e-8 * np.linalg.norm(f) * (1 + 1e-6)
    assert st["iface_iterations"] >= st["iterations"]
    h = st["history"]
    assert len(h) == st["iterations"] + 1 and h[0] == 1.0 and h[-1] <= 1e-8 * (1 + 1e-6)
    # the oracle's flexible outer PCG with its FP32 inexact interface solve
    ii = oi.inexact_setup(pc, 2, np.float32)
    ref = oa.pcg(A, f, lambda r: oi.apply_inexact(pc, ii, r, rtol=1e-2), tol=1e-8, flexible=True)
    exact = oa.pcg(A, f, lambda r: oa.apply(pc, r), tol=1e-8)
    assert ref.converged
    assert abs(st["iterations"] - ref.iterations) <= max(3, ref.iterations // 10)
    assert st["iterations"] >= exact.iterations - 1


def test_graph_replay_and_stage_times(case):
    """The cluster launch replays inside the captured iteration graph with bit-identical
    results; per-stage times (stream-ordered run) come back for the last iteration."""
    A, f, sizes, part, pc = case
    a = AM(A, sizes, use_graph=False)
    b = AM(A, sizes, use_graph=True, check_every=3)
    c = AM(A, sizes, use_graph=True, stage_times=True)
    xa, sa = a.solve(f, tol=1e-9)
    xb, sb = b.solve(f, tol=1e-9)
    xc, sc = c.solve(f, tol=1e-9)
    assert sa["iterations"] == sb["iterations"] == sc["iterations"]
    assert torch.equal(xa, xb) and torch.equal(xa, xc)
    assert all(v > 0 for v in sc["stage_ms"].values())
    assert all(v == 0 for v in sa["stage_ms"].values())


def test_multi_rhs(case):
    A, f, sizes, part, pc = case
    am = AM(A, sizes)
    rng = np.random.default_rng(9)
    Bm = np.stack([f] + [rng.standard_normal(A.shape[0]) for _ in range(2)], axis=1)
    X, sts = am.solve_multi(Bm, tol=1e-8)
    X = X.cpu().numpy()
    for j in range(3):
        assert sts[j]["status"] == 0
        assert np.linalg.norm(Bm[:, j] - A @ X[:, j]) <= 1e-8 * np.linalg.norm(Bm[:, j]) * (1 + 1e-6)
        assert sts[j]["iface_iterations"] >= sts[j]["iterations"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_low_precision_with_inexact_interface(case, prec):
    A, f, sizes, part, pc = case
    am = AM(A, sizes, precision=prec)
    x, st = am.solve(f, tol=1e-8)
    assert st["status"] == 0
    assert np.linalg.norm(f - A @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(f) * (1 + 1e-6)


def test_oversized_block_is_rejected():
    """60 subdomains, 312 interfaces: one block of all of them exceeds the 128-interface
    limit of the block-Jacobi inverses and setup says so."""
    lnK = synth.gaussian_field((21, 17, 13), 3.0, 2.0, 31)
    A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=1)
    sizes = synth.even_part_sizes(A.shape[0], 60)
    from paper_2607_22905_b300 import binding as B
    with pytest.raises(B.AlgMortarError, match="block-Jacobi block"):
        AM(A, sizes, iface_block_parts=100000)
    am = AM(A, sizes, iface_block_parts=4)
    x, st = am.solve(f, tol=1e-8)
    assert st["status"] == 0


def test_noalloc_entry_point_refuses_inexact(case):
    A, f, sizes, part, pc = case
    am = AM(A, sizes)
    from paper_2607_22905_b300 import binding as B
    import ctypes as C
    L = am.info["n_lambda"]
    b = torch.zeros(L, dtype=torch.float64, device="cuda")
    e = torch.zeros_like(b)
    rc = B.lib().algmortar_interface_solve_noalloc(am._h, C.c_void_p(b.data_ptr()), C.c_void_p(e.data_ptr()))
    assert rc == B.INVALID_ARG
