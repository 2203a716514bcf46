"""The workloads at their full sizes, in the launch configuration bench.py times.

Config 3 (1.122M cells) gets a complete oracle comparison of the preconditioner (the
oracle's Algorithm 1/2 takes ~20 s there); PCG results are checked through the true
residual; configs 2, 4 and 5 through properties that hold at any size (true residual,
symmetry, the Sec. 5.4 residual structure, a directional finite difference of the
adjoint gradient).
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


@pytest.fixture(scope="module")
def c3():
    return synth.config3()


def test_c3_apply_matches_oracle(c3):
    P = c3
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision="fp64", use_graph=True, check_every=8)
    part = op.partition(P.A, P.part_sizes)
    np.testing.assert_array_equal(am.partition(), part)
    pc = oa.setup(P.A, part)
    r = np.random.default_rng(3).standard_normal(P.n)
    z = am.apply(r).cpu().numpy()
    zo = oa.apply(pc, r)
    assert rel(z, zo) <= 1e-10
    assert rel_sub(z, zo, part) <= 1e-10
    pbar, beta, eta, _ = am.apply_stages(r)
    pbar_o, rhs_o, eta_o, _ = oa.apply_parts(pc, r)
    orig, orig_o = np.empty(P.n), np.empty(P.n)
    orig[am.permutation()] = pbar.cpu().numpy()
    orig_o[pc.sk.perm] = pbar_o
    assert rel(orig, orig_o) <= 1e-10
    assert rel_sub(orig, orig_o, part) <= 1e-10
    assert rel(beta.cpu().numpy(), rhs_o) <= 1e-10
    assert rel(eta.cpu().numpy(), eta_o) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_c3_pcg_converges(c3, precision):
    P = c3
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=precision, use_graph=True, check_every=8)
    x, st = am.solve(P.f, tol=1e-8)
    x = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(P.f - P.A @ x) <= 1e-8 * np.linalg.norm(P.f)
    r1, r2 = np.random.default_rng(4).standard_normal((2, P.n))
    a = float(r1 @ am.apply(r2).cpu().numpy())
    b = float(r2 @ am.apply(r1).cpu().numpy())
    # FP64: symmetric to rounding; low-precision factors: the solve L^-T L^-1 still is
    assert abs(a - b) <= (1e-12 if precision == "fp64" else 1e-6) * (abs(a) + abs(b))


def test_c2_end_to_end():
    P = synth.config2()
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision="fp32", use_graph=True, check_every=8)
    x, st = am.solve(P.f, tol=1e-8)
    x = x.cpu().numpy()
    assert st["status"] == 0
    assert np.linalg.norm(P.f - P.A @ x) <= 1e-8 * np.linalg.norm(P.f)
    # Sec. 5.4 residual structure with the FP64 preconditioner at full size
    am64 = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision="fp64")
    r = np.random.default_rng(5).standard_normal(P.n)
    z = am64.apply(r).cpu().numpy()
    res = r - P.A @ z
    part = am64.partition()
    coo = sp.coo_matrix(P.A)
    iface = np.zeros(P.n, dtype=bool)
    iface[coo.row[part[coo.row] != part[coo.col]]] = True
    assert np.abs(res[~iface]).max() <= 1e-9 * np.abs(r).max()


def test_c4_faulted_multi_rhs():
    P = synth.config4()
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision="fp32", use_graph=True, check_every=8)
    B = P.meta["rhs"][:, :4]
    X, stats = am.solve_multi(B, tol=1e-8)
    X = X.cpu().numpy()
    for j in range(B.shape[1]):
        assert stats[j]["status"] == 0
        assert np.linalg.norm(B[:, j] - P.A @ X[:, j]) <= 1e-8 * np.linalg.norm(B[:, j])
    # the single-RHS solve of a column agrees to the tolerance (the batched local solve
    # sums in another order)
    x0, st0 = am.solve(B[:, 0], tol=1e-8)
    x0 = x0.cpu().numpy()
    assert np.linalg.norm(x0 - X[:, 0]) <= 1e-6 * np.linalg.norm(x0)
    assert abs(st0["iterations"] - stats[0]["iterations"]) <= 2


def test_c5_adjoint_directional_fd():
    """96^3, ln K ~ N(0, 2^2): the adjoint gradient against a central difference of the
    misfit along a random direction (GPU solves at 1e-12)."""
    from paper_2607_22905_b300.adjoint import AlgMortarTPFASolve
    n = 96
    shape = (n, n, n)
    lnK = synth.gaussian_field(shape, 6.0, 2.0, 50)
    A, f, faces = synth.tpfa_from_lnK(lnK)
    am = AlgMortar(A, A.shape[0] // 1728, precision="bf16", use_graph=True, check_every=8)
    x_ref, _ = am.solve(f, tol=1e-10)
    obs, p_obs = synth.observations(A.shape[0], 200, 5001, x_ref.cpu().numpy() * 0.9)

    def assemble(t):
        Ah, fh, fc = synth.tpfa_from_lnK(t.cpu().numpy().reshape(shape, order="F"))
        tb, tbp = synth.tpfa_cell_bc(Ah.shape[0], fc)
        return Ah.data, fh, tb, tbp

    o = torch.as_tensor(obs, device="cuda")
    po = torch.as_tensor(p_obs, device="cuda")
    flat = torch.tensor(lnK.ravel(order="F"), device="cuda", requires_grad=True)
    p = AlgMortarTPFASolve.apply(flat, am, assemble, 1e-12)
    loss = ((p[o] - po) ** 2).sum()
    loss.backward()
    g = flat.grad
    d = torch.as_tensor(np.random.default_rng(6).standard_normal(flat.numel()), device="cuda")
    h = 1e-5
    vals = []
    for s in (1, -1):
        ps = AlgMortarTPFASolve.apply((flat.detach() + s * h * d), am, assemble, 1e-12)
        vals.append(float(((ps[o] - po) ** 2).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    gd = float((g * d).sum())
    assert abs(fd - gd) <= 1e-4 * abs(gd)
