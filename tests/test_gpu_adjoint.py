"""Hand-written adjoint through AlgMortar-PCG (config 5 workload, reduced sizes), through
the C ABI, against the oracle's dense-solve gradient and central finite differences."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import synth
from oracle import adjoint as oadj

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_22905_b300 import build
    build.build()


def problem(n, seed, n_obs, ref_seed=5999):
    shape = (n, n, n)
    lnK = synth.gaussian_field(shape, 6.0, 2.0, seed)
    A, f, faces = synth.tpfa_from_lnK(lnK)
    lnK_ref = synth.gaussian_field(shape, 6.0, 2.0, ref_seed)
    Ar, fr, _ = synth.tpfa_from_lnK(lnK_ref)
    p_ref = spla.spsolve(Ar.tocsc(), fr)
    obs, p_obs = synth.observations(A.shape[0], n_obs, 5001, p_ref)
    return shape, lnK, A, f, faces, obs, p_obs


def assembler(shape):
    def assemble(lnK_t):
        lnK = lnK_t.cpu().numpy().reshape(shape, order="F")
        A, f, faces = synth.tpfa_from_lnK(lnK)
        tb, tbp = synth.tpfa_cell_bc(A.shape[0], faces)
        return A.data, f, tb, tbp
    return assemble


def gpu_grad(solver, shape, lnK, obs, p_obs, tol):
    from paper_2607_22905_b300.adjoint import AlgMortarTPFASolve
    x = torch.tensor(lnK.ravel(order="F"), dtype=torch.float64, device="cuda", requires_grad=True)
    p = AlgMortarTPFASolve.apply(x, solver, assembler(shape), tol)
    o = torch.as_tensor(obs, device="cuda")
    loss = ((p[o] - torch.as_tensor(p_obs, device="cuda")) ** 2).sum()
    loss.backward()
    return float(loss), x.grad.cpu().numpy()


def dense_solve(M, v):
    return sla.cho_solve(sla.cho_factor(M.toarray()), v)


def test_adjoint_matches_dense_reference_and_fd():
    from paper_2607_22905_b300.solver import AlgMortar
    shape, lnK, A, f, faces, obs, p_obs = problem(16, 50, 200)
    solver = AlgMortar(A, 8)
    L, g = gpu_grad(solver, shape, lnK, obs, p_obs, 1e-13)
    Lr, gr, _, _ = oadj.grad_lnK(A, f, faces, lnK.ravel(order="F"), obs, p_obs, dense_solve)
    assert abs(L - Lr) <= 1e-9 * abs(Lr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
    # central finite differences (h = 1e-6) with dense solves on 64 seeded entries
    flat = lnK.ravel(order="F")
    rng = np.random.default_rng(7)
    h = 1e-6
    for k in rng.choice(flat.size, 64, replace=False):
        vals = []
        for sgn in (1, -1):
            q = flat.copy()
            q[k] += sgn * h
            Ah, fh, _ = synth.tpfa_from_lnK(q.reshape(shape, order="F"))
            vals.append(oadj.misfit(dense_solve(Ah, fh), obs, p_obs))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * np.abs(g).max()


def test_adjoint_batch_of_samples_one_handle():
    """8 permeability samples (seeds 50-57) through one handle (value updates), each
    gradient equal to the oracle's sparse-direct adjoint gradient."""
    from paper_2607_22905_b300.solver import AlgMortar
    n = 24
    shape, lnK0, A0, *_ = problem(n, 50, 200)
    solver = AlgMortar(A0, 16, precision="fp64", use_graph=True)
    sp_solve = lambda M, v: spla.spsolve(M.tocsc(), v)
    for seed in range(50, 58):
        shape, lnK, A, f, faces, obs, p_obs = problem(n, seed, 200)
        L, g = gpu_grad(solver, shape, lnK, obs, p_obs, 1e-12)
        Lr, gr, _, _ = oadj.grad_lnK(A, f, faces, lnK.ravel(order="F"), obs, p_obs, sp_solve)
        assert abs(L - Lr) <= 1e-8 * abs(Lr)
        assert np.linalg.norm(g - gr) <= 1e-7 * np.linalg.norm(gr)


def test_adjoint_mixed_precision_factors():
    """BF16 local factors: same gradient to the solve tolerance (the preconditioner
    changes, the converged solves do not)."""
    from paper_2607_22905_b300.solver import AlgMortar
    shape, lnK, A, f, faces, obs, p_obs = problem(16, 51, 200)
    _, g64 = gpu_grad(AlgMortar(A, 8), shape, lnK, obs, p_obs, 1e-12)
    _, g16 = gpu_grad(AlgMortar(A, 8, precision="bf16"), shape, lnK, obs, p_obs, 1e-12)
    assert np.linalg.norm(g16 - g64) <= 1e-7 * np.linalg.norm(g64)
