"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 factors -> preconditioned vectors agree to 1e-10 relative (the stated
FP64 bar; both sides are backward-stable solves of the same SPD systems, so the
difference is a few ulps times the local condition numbers); solutions agree within the
solve tolerance.  FP32 / BF16 factors change the preconditioner itself, so for them the
checks are convergence to the same tolerance and closeness of the solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import algmortar as oa
from oracle import partition as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_22905_b300 import build
    build.build()


def AlgMortar(*a, **k):
    from paper_2607_22905_b300.solver import AlgMortar as _A
    return _A(*a, **k)


def rel(a, b):
    """Worse of the norm-wise error and the element-wise one, max |a - b| / max |b|."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    nb = max(float(np.linalg.norm(b)), 1e-300)
    mb = max(float(np.abs(b).max(initial=0.0)), 1e-300)
    return max(float(np.linalg.norm(d)) / nb, float(d.max(initial=0.0)) / mb)


def rel_sub(a, b, labels):
    """Largest norm-wise error over the subdomains (labels: subdomain of each entry), so
    that a wrong value in a small-magnitude subdomain cannot hide under the others."""
    a, b, labels = np.asarray(a), np.asarray(b), np.asarray(labels)
    worst = 0.0
    for s in np.unique(labels):
        sel = labels == s
        worst = max(worst, float(np.linalg.norm(a[sel] - b[sel]) / max(np.linalg.norm(b[sel]), 1e-300)))
    return worst


def small3d(shape=(21, 17, 13), m=11, seed=31, uneven=True, sigma=2.0):
    """3D TPFA with ragged subdomains (sizes not multiples of the 32-row tile)."""
    lnK = synth.gaussian_field(shape, 3.0, sigma, seed)
    A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=1)
    n = A.shape[0]
    sizes = synth.uneven_part_sizes(n, m, 150, 900, seed) if uneven else synth.even_part_sizes(n, m)
    return A, f, sizes


CASES = {
    "c1": lambda: (lambda P: (P.A, P.f, P.part_sizes))(synth.config1()),
    "3d_uneven": lambda: small3d(),
    "3d_even_ragged": lambda: small3d(shape=(19, 15, 11), m=8, uneven=False, seed=7),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    A, f, sizes = CASES[request.param]()
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    return request.param, A, f, sizes, part, pc


def test_partition_and_permutation(case):
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    np.testing.assert_array_equal(am.partition(), part)
    perm = am.permutation()
    assert sorted(perm.tolist()) == list(range(A.shape[0]))
    # the internal ordering groups subdomains in order
    assert (np.diff(part[perm]) >= 0).all()
    np.testing.assert_array_equal(am.interfaces(), pc.sk.pairs)


def test_apply_fp64_matches_oracle(case):
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    rng = np.random.default_rng(100)
    for _ in range(3):
        r = rng.standard_normal(A.shape[0])
        z = am.apply(r).cpu().numpy()
        zo = oa.apply(pc, r)
        assert rel(z, zo) <= 1e-10
        assert rel_sub(z, zo, part) <= 1e-10


def test_apply_stages_fp64(case):
    """Each stage of Algorithm 2: pbar (Eq. def-pbar-local), interface RHS, eta, z."""
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    r = np.random.default_rng(101).standard_normal(A.shape[0])
    pbar, beta, eta, z = (t.cpu().numpy() for t in am.apply_stages(r))
    perm = am.permutation()                      # internal -> original
    pbar_o, rhs_o, eta_o, z_o = oa.apply_parts(pc, r)
    # oracle vectors are in its own (part, index) ordering: map both to original
    orig_pbar = np.empty_like(pbar)
    orig_pbar[perm] = pbar
    orig_pbar_o = np.empty_like(pbar_o)
    orig_pbar_o[pc.sk.perm] = pbar_o
    assert rel(orig_pbar, orig_pbar_o) <= 1e-10
    assert rel_sub(orig_pbar, orig_pbar_o, part) <= 1e-10
    assert rel(beta, rhs_o) <= 1e-10
    assert rel(eta, eta_o) <= 1e-10
    orig_z = np.empty_like(z)
    orig_z[perm] = z
    orig_z_o = np.empty_like(z_o)
    orig_z_o[pc.sk.perm] = z_o
    assert rel(orig_z, orig_z_o) <= 1e-10
    assert rel_sub(orig_z, orig_z_o, part) <= 1e-10


def test_apply_symmetric(case):
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    rng = np.random.default_rng(102)
    r1, r2 = rng.standard_normal((2, A.shape[0]))
    a = float(r1 @ am.apply(r2).cpu().numpy())
    b = float(r2 @ am.apply(r1).cpu().numpy())
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_residual_vanishes_off_interface(case):
    """Sec. 5.4 on the GPU result: r - A z is zero at cells without interface edges."""
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    r = np.random.default_rng(103).standard_normal(A.shape[0])
    z = am.apply(r).cpu().numpy()
    res = r - A @ z
    coo = sp.coo_matrix(A)
    iface = np.zeros(A.shape[0], dtype=bool)
    cross = part[coo.row] != part[coo.col]
    iface[coo.row[cross]] = True
    assert np.abs(res[~iface]).max() <= 1e-10 * np.abs(r).max()


@pytest.mark.parametrize("use_graph", [False, True])
def test_pcg_fp64_matches_oracle(case, use_graph):
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes, use_graph=use_graph, check_every=4 if use_graph else 1)
    x, st = am.solve(f, tol=1e-8)
    x = x.cpu().numpy()
    ref = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-8)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    assert np.linalg.norm(f - A @ x) <= 1e-8 * np.linalg.norm(f)
    assert abs(st["iterations"] - ref.iterations) <= 1
    xs = spla.spsolve(A.tocsc(), f)
    assert rel(x, ref.x) <= 1e-6 and rel(x, xs) <= 1e-6


def test_graph_and_stream_paths_bitwise_equal(case):
    name, A, f, sizes, part, pc = case
    a = AlgMortar(A, len(sizes), part_sizes=sizes)
    b = AlgMortar(A, len(sizes), part_sizes=sizes, use_graph=True, check_every=1)
    xa, sa = a.solve(f)
    xb, sb = b.solve(f)
    assert sa["iterations"] == sb["iterations"]
    assert torch.equal(xa, xb)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pcg_low_precision_factors(case, precision):
    """Mixed precision: local factors in FP32/BF16, outer PCG FP64 -> same tolerance."""
    name, A, f, sizes, part, pc = case
    am = AlgMortar(A, len(sizes), part_sizes=sizes, precision=precision)
    x, st = am.solve(f, tol=1e-8)
    x = x.cpu().numpy()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-8
    ref = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-8)
    assert rel(x, ref.x) <= 1e-5
    assert st["iterations"] <= 2 * ref.iterations + 5
    # the low-precision preconditioner stays close to the FP64 one
    r = np.random.default_rng(104).standard_normal(A.shape[0])
    tol = 2e-3 if precision == "fp32" else 1e-1
    assert rel(am.apply(r).cpu().numpy(), oa.apply(pc, r)) <= tol


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("depth", [0, 2])
def test_low_precision_variants_apply_the_interface_inverses_in_fp32(precision, depth):
    """FP32 / BF16 factor variants apply the explicit interface inverses in FP32: eta
    against the oracle's exact solve of S_eta with the GPU's own b_eta.  The handle's S_eta
    is built from MBFs solved with its own factors, so it matches the exact S_eta to FP32
    rounding for FP32 factors and only to BF16 rounding (~1e-2) for BF16 factors."""
    A, f, sizes = small3d(shape=(23, 19, 15), m=16, seed=41)
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    am = AlgMortar(A, len(sizes), part_sizes=sizes, nd_depth=depth, precision=precision)
    r = np.random.default_rng(107).standard_normal(A.shape[0])
    _, beta, eta, _ = (t.cpu().numpy() for t in am.apply_stages(r))
    eta_ref = np.linalg.solve(pc.S, beta)
    assert rel(eta, eta_ref) <= (1e-4 if precision == "fp32" else 5e-2)
    x, st = am.solve(f, tol=1e-8)
    assert st["status"] == 0


@pytest.mark.parametrize("depth", [0, 1, 2])
def test_interface_nested_dissection(depth):
    """The interface solve by nested dissection (2^depth groups + separator) gives the
    same eta and z as the oracle's dense Cholesky of S_eta."""
    A, f, sizes = small3d(shape=(23, 19, 15), m=16, seed=41)
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    am = AlgMortar(A, len(sizes), part_sizes=sizes, nd_depth=depth)
    r = np.random.default_rng(106).standard_normal(A.shape[0])
    pbar, beta, eta, z = (t.cpu().numpy() for t in am.apply_stages(r))
    _, rhs_o, eta_o, _ = oa.apply_parts(pc, r)
    assert rel(beta, rhs_o) <= 1e-10
    assert rel(eta, eta_o) <= 1e-10
    assert rel(am.apply(r).cpu().numpy(), oa.apply(pc, r)) <= 1e-10
    x, st = am.solve(f, tol=1e-8)
    ref = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-8)
    assert st["status"] == 0 and abs(st["iterations"] - ref.iterations) <= 1


def test_update_values_matches_fresh_setup():
    """New values on the same pattern (a second permeability sample) through
    algmortar_update_values equal a fresh setup, for the host and device paths."""
    A, f, sizes = small3d(seed=31)
    A2, f2, _ = small3d(seed=32)
    assert (A.indices == A2.indices).all() and (A.indptr == A2.indptr).all()
    am = AlgMortar(A, len(sizes), part_sizes=sizes, use_graph=True)
    x1, _ = am.solve(f)
    fresh = AlgMortar(A2, len(sizes), part_sizes=sizes)
    for vals in (A2.data, torch.as_tensor(A2.data, device="cuda")):
        am.update_values(vals)
        xa, sa = am.solve(f2)
        xb, sb = fresh.solve(f2)
        assert sa["iterations"] == sb["iterations"]
        assert torch.equal(xa, xb)


def test_single_subdomain_exact():
    """m = 1: no interface, z = A^{-1} r; PCG converges in one iteration."""
    A, f, _ = small3d(shape=(9, 8, 7), m=1, uneven=False)
    am = AlgMortar(A, 1)
    assert am.info["n_lambda"] == 0
    r = np.random.default_rng(105).standard_normal(A.shape[0])
    x = spla.spsolve(A.tocsc(), r)
    assert rel(am.apply(r).cpu().numpy(), x) <= 1e-11
    xs, st = am.solve(f, tol=1e-10)
    assert st["iterations"] == 1


def test_solve_host_matches_device():
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    xd, sd = am.solve(f)
    xh, sh = am.solve_host(f)
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)
    assert sd["iterations"] == sh["iterations"]


def test_zero_rhs():
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes)
    x, st = am.solve(np.zeros(A.shape[0]))
    assert st["iterations"] == 0 and float(x.abs().max()) == 0.0


def test_max_it_reports_no_convergence():
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes, max_it=3)
    x, st = am.solve(f, tol=1e-12, raise_on_fail=False)
    assert st["status"] == 5 and st["iterations"] == 3


@pytest.mark.parametrize("use_graph", [False, True])
def test_multi_rhs_batches_bitwise_equal_single(use_graph):
    """35 right-hand sides (a batch of 32 and a ragged batch of 3; column blocks of 4 with a
    ragged last block): every column converges on its own, agrees with the single-RHS
    solve to the tolerance with the same iteration count to +-2; a zero column stops at
    once, a column scaled by 1e6 takes its own path."""
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes, precision="fp32", use_graph=use_graph, check_every=3)
    rng = np.random.default_rng(12)
    k = 35
    Bm = rng.standard_normal((A.shape[0], k))
    Bm[:, 3] = 0.0
    Bm[:, 4] *= 1e6
    Bm[:, 5] = f
    X, stats = am.solve_multi(Bm, tol=1e-9)
    its = set()
    for j in range(k):
        x, st = am.solve(Bm[:, j], tol=1e-9)
        if j != 3:
            assert rel(X[:, j].cpu().numpy(), x.cpu().numpy()) <= 1e-6, j
        assert abs(stats[j]["iterations"] - st["iterations"]) <= 2
        assert stats[j]["status"] == 0
        its.add(st["iterations"])
        if j != 3:
            xj = X[:, j].cpu().numpy()
            assert np.linalg.norm(Bm[:, j] - A @ xj) <= 1e-9 * np.linalg.norm(Bm[:, j])
    assert stats[3]["iterations"] == 0 and float(X[:, 3].abs().max()) == 0.0
    assert len(its) > 1


def test_multi_rhs_matches_oracle_pcg():
    """Batched FP64 solves against the oracle's PCG on the same seeded columns."""
    A, f, sizes = small3d(shape=(19, 15, 11), m=8, uneven=False, seed=7)
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    am = AlgMortar(A, len(sizes), part_sizes=sizes, precision="fp64")
    Bm = np.random.default_rng(13).standard_normal((A.shape[0], 4))
    X, stats = am.solve_multi(Bm, tol=1e-10)
    for j in range(4):
        ref = oa.pcg(A, Bm[:, j], lambda v: oa.apply(pc, v), 1e-10)
        assert abs(stats[j]["iterations"] - ref.iterations) <= 1
        assert rel(X[:, j].cpu().numpy(), ref.x) <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_flexible_beta(precision):
    """Polak-Ribiere beta: with the FP64 (symmetric) preconditioner r_{k+1}.z_k = 0 in
    exact arithmetic, so the iteration count matches the standard beta to +-1; with
    low-precision factors it converges to the same tolerance."""
    A, f, sizes = small3d()
    std = AlgMortar(A, len(sizes), part_sizes=sizes, precision=precision)
    flx = AlgMortar(A, len(sizes), part_sizes=sizes, precision=precision, flexible=True, use_graph=True,
                    check_every=4)
    xs, ss = std.solve(f, tol=1e-10)
    xf, sf = flx.solve(f, tol=1e-10)
    assert sf["status"] == 0
    assert np.linalg.norm(f - A @ xf.cpu().numpy()) <= 1e-10 * np.linalg.norm(f)
    if precision == "fp64":
        assert abs(sf["iterations"] - ss["iterations"]) <= 1
    else:
        assert sf["iterations"] <= ss["iterations"] + 3


def test_tight_tolerance_reports_true_residual():
    """A tolerance near the FP64 floor with BF16 factors: the solver either confirms it on
    the true residual (after residual replacements) or reports NO_CONVERGENCE; it never
    breaks down, and the reported residual is the true one."""
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes, precision="bf16", use_graph=True, check_every=4)
    x, st = am.solve(f, tol=1e-14, raise_on_fail=False)
    assert st["status"] in (0, 5)
    true = np.linalg.norm(f - A @ x.cpu().numpy()) / np.linalg.norm(f)
    assert abs(true - st["rel_residual"]) <= 1e-3 * true + 1e-16


def test_wide_profile_many_tiles_per_row():
    """Two subdomains of ~2300 cells (73 tile rows, ~3 off-diagonal tiles per row): each
    chain streams ~8 times its ring's capacity, so ring slots are reused while tiles are
    released out of order by different warps.  FP64 apply matches the oracle; the
    autotuned launch variant agrees to rounding;
    FP32 / BF16 PCG converge."""
    A, f, sizes = small3d(m=2, uneven=False)
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    r = np.random.default_rng(21).standard_normal(A.shape[0])
    z_ref = oa.apply(pc, r)
    for prec in ("fp64", "fp32", "bf16"):
        am = AlgMortar(A, len(sizes), part_sizes=sizes, precision=prec)
        tuned = AlgMortar(A, len(sizes), part_sizes=sizes, precision=prec, autotune=True)
        z = am.apply(r)
        assert rel(tuned.apply(r).cpu().numpy(), z.cpu().numpy()) <= (1e-13 if prec == "fp64" else 1e-6)
        if prec == "fp64":
            assert rel(z.cpu().numpy(), z_ref) <= 1e-10
        else:
            assert rel(z.cpu().numpy(), z_ref) <= (1e-4 if prec == "fp32" else 3e-2)
        x, st = am.solve(f, tol=1e-9)
        assert st["status"] == 0
        assert np.linalg.norm(f - A @ x.cpu().numpy()) <= 1e-9 * np.linalg.norm(f)


@pytest.mark.parametrize("nu", [1, 2])
def test_smoothed_apply_matches_oracle(nu):
    """Block-Jacobi pre/post smoothing (Sec. 5.4), FP64: the composite preconditioner
    against the oracle's, element by element, and PCG with fewer iterations than nu = 0."""
    from oracle import smoothing as osm
    A, f, sizes = small3d()
    part = op.partition(A, sizes)
    pc = oa.setup(A, part)
    bj = osm.block_jacobi_setup(A, part)
    am = AlgMortar(A, len(sizes), part_sizes=sizes, smooth_steps=nu, use_graph=True, check_every=2)
    rng = np.random.default_rng(30 + nu)
    for _ in range(2):
        r = rng.standard_normal(A.shape[0])
        assert rel(am.apply(r).cpu().numpy(), osm.smoothed_apply(A, pc, bj, r, nu)) <= 1e-10
    x, st = am.solve(f, tol=1e-8)
    assert st["status"] == 0
    ref = oa.pcg(A, f, lambda v: osm.smoothed_apply(A, pc, bj, v, nu), 1e-8)
    assert abs(st["iterations"] - ref.iterations) <= 1
    x0, st0 = AlgMortar(A, len(sizes), part_sizes=sizes).solve(f, tol=1e-8)
    assert st["iterations"] < st0["iterations"]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_smoothed_low_precision_and_multi_rhs(precision):
    """Smoothing with low-precision factors converges; batched columns agree with the
    single-RHS solves to the tolerance."""
    A, f, sizes = small3d()
    am = AlgMortar(A, len(sizes), part_sizes=sizes, precision=precision, smooth_steps=1, use_graph=True,
                   check_every=3)
    Bm = np.random.default_rng(40).standard_normal((A.shape[0], 3))
    X, stats = am.solve_multi(Bm, tol=1e-9)
    for j in range(3):
        x, st = am.solve(Bm[:, j], tol=1e-9)
        assert rel(X[:, j].cpu().numpy(), x.cpu().numpy()) <= 1e-6
        assert stats[j]["status"] == 0
        assert np.linalg.norm(Bm[:, j] - A @ x.cpu().numpy()) <= 1e-9 * np.linalg.norm(Bm[:, j])


def _pair_edge_cases():
    # checkerboard colouring: no coupling inside a subdomain, so every local block is
    # diagonal (no off-diagonal tiles at all) and each chain has 25 tile rows (odd)
    A1, f1 = synth.tpfa_cartesian(np.exp(synth.gaussian_field((40, 40, 1), 3.0, 1.0, 3)), bc_axis=0)
    ii, jj = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    chk = ((ii + jj) % 2).ravel(order="F").astype(np.int32)
    # parts of 1, 2, 3 and 5 tile rows (20, 45, 90, 150 cells) on a 61 x 5 strip
    A2, f2 = synth.tpfa_cartesian(np.exp(synth.gaussian_field((61, 5, 1), 3.0, 1.0, 4)), bc_axis=0)
    # a 1D chain of 700 cells in 2 parts (bandwidth-1 factors, 11 tile rows each)
    A3, f3 = synth.tpfa_cartesian(np.exp(synth.gaussian_field((700, 1, 1), 5.0, 1.0, 5)), bc_axis=0)
    # a part of a single cell (one tile row holding one row) next to a large one
    A4, f4 = synth.tpfa_cartesian(np.exp(synth.gaussian_field((12, 10, 3), 3.0, 1.0, 6)), bc_axis=0)
    lab4 = np.zeros(A4.shape[0], dtype=np.int32)
    lab4[0] = 1
    # a hub subdomain (the middle row of a 70 x 21 grid) with 70 neighbours: more
    # interfaces than the prolongation holds in lane registers (64)
    K5 = np.exp(synth.gaussian_field((70, 21, 1), 3.0, 1.0, 8))
    A5, f5 = synth.tpfa_cartesian(K5, bc_axis=0)
    idx5 = synth.cell_index(K5.shape)
    lab5 = np.empty(A5.shape[0], dtype=np.int32)
    for x in range(70):
        for y in range(21):
            lab5[idx5[x, y, 0]] = 0 if y == 10 else (1 + x // 2 if y < 10 else 36 + x // 2)
    return {"checkerboard": (A1, f1, chk, None), "tiny_parts": (A2, f2, None, [20, 45, 90, 150]),
            "chain": (A3, f3, None, [350, 350]), "one_cell_part": (A4, f4, lab4, None),
            "hub_70_interfaces": (A5, f5, lab5, None)}


@pytest.mark.parametrize("name", ["checkerboard", "tiny_parts", "chain", "one_cell_part", "hub_70_interfaces"])
def test_pair_chain_edge_profiles(name):
    """Edge cases of the paired tile rows (FP32/BF16): chains of 1-5 tile rows (odd counts
    end on a single row), and diagonal local blocks (no near, far or coupling tiles).
    FP64 apply matches the oracle; FP32/BF16 applies stay close to it and are symmetric
    to rounding (the backward stream is the exact transpose of the forward one); PCG
    converges for all three."""
    A, f, labels, sizes = _pair_edge_cases()[name]
    if labels is None:
        part = op.partition(A, sizes)
        m = len(sizes)
    else:
        part = labels
        m = int(labels.max()) + 1
    pc = oa.setup(A, part)
    # condition of the diagonally scaled local blocks (the factored matrices)
    kappa = max(np.linalg.cond(Ai.toarray() / np.sqrt(np.outer(Ai.diagonal(), Ai.diagonal())))
                for Ai in pc.A_loc)
    # a relative perturbation of S_eta (built from the low-precision MBFs) reaches eta
    # amplified by the condition of the scaled interface matrix
    if pc.S.size:
        d = np.sqrt(np.diag(pc.S))
        kappa *= max(1.0, float(np.linalg.cond(pc.S / np.outer(d, d))))
    rng = np.random.default_rng(77)
    r, s2 = rng.standard_normal((2, A.shape[0]))
    z_ref = oa.apply(pc, r)
    for prec in ("fp64", "fp32", "bf16"):
        am = AlgMortar(A, m, parts=part, precision=prec)
        z = am.apply(r).cpu().numpy()
        if prec == "fp64":
            assert rel(z, z_ref) <= 1e-10
        else:
            # low-precision factors perturb the preconditioner by ~cond(A_i) cond(S_eta) *
            # unit roundoff (FP32 2^-24, BF16 2^-9): compared where that leaves the
            # comparison meaningful (bounds of test_pcg_low_precision_factors)
            u, bound = (2.0 ** -24, 2e-3) if prec == "fp32" else (2.0 ** -9, 1e-1)
            if 4 * kappa * u <= bound:
                assert rel(z, z_ref) <= bound
            # symmetric up to the FP32 rounding of the solve's accumulations, measured on
            # the Cauchy-Schwarz scale of the bilinear form
            a_ = float(s2 @ z)
            b_ = float(r @ am.apply(s2).cpu().numpy())
            assert abs(a_ - b_) <= 1e-6 * np.linalg.norm(s2) * np.linalg.norm(z)
        x, st = am.solve(f, tol=1e-9)
        assert st["status"] == 0
        assert np.linalg.norm(f - A @ x.cpu().numpy()) <= 1e-9 * np.linalg.norm(f)
