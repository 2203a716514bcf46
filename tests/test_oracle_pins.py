"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks an identity, a closed form,
an independent assembly, a library solve or brute force.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import adjoint as oadj
from oracle import algmortar as oa
from oracle import partition as op

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(shape=(8, 6, 1), sigma=1.0, seed=11, m=4):
    lnK = synth.gaussian_field(shape, 2.0, sigma, seed)
    A, f = synth.tpfa_cartesian(np.exp(lnK), bc_axis=0)
    part = op.partition(A, synth.even_part_sizes(A.shape[0], m))
    return A, f, part


def dense_ops(pc):
    return (pc.W.toarray(), pc.M.toarray(), pc.B.toarray(), pc.Z.toarray(),
            sp.block_diag(pc.A_loc).toarray(), pc.sk.A.toarray())


@pytest.fixture(scope="module")
def p2d():
    A, f, part = small_problem()
    return A, f, part, oa.setup(A, part)


@pytest.fixture(scope="module")
def p3d():
    A, f, part = small_problem(shape=(6, 5, 4), sigma=1.5, seed=5, m=6)
    return A, f, part, oa.setup(A, part)


# ------------------------------------------------------------------ operators (Sec. 3.2)

def test_prop_BWM(p2d, p3d):
    """Prop. proposition-BWM: B^T = 4 W M, exactly."""
    for *_, pc in (p2d, p3d):
        W, M, B, *_ = dense_ops(pc)
        np.testing.assert_array_equal(B.T, 4.0 * W @ M)


def test_trace_identities(p3d):
    """Eqs. (UWL-identity), (LWL-identity), (UWU-identity) on random p."""
    *_, pc = p3d
    sk = pc.sk
    W, L, U, M, B, Z = oa.operators(sk)
    rng = np.random.default_rng(0)
    p = rng.standard_normal(sk.n)
    s_uwl = np.sum(sk.ea * p[sk.ek] * p[sk.el])
    s_lwl = np.sum(sk.ea * p[sk.ek] ** 2)
    s_uwu = np.sum(sk.ea * p[sk.el] ** 2)
    assert np.isclose(p @ (U.T @ (W @ (L @ p))), s_uwl, rtol=1e-13)
    assert np.isclose(p @ (L.T @ (W @ (L @ p))), s_lwl, rtol=1e-13)
    assert np.isclose(p @ (U.T @ (W @ (U @ p))), s_uwu, rtol=1e-13)
    # (M p)_e = (p_k + p_l)/2, Eq. (global-edge-repr)
    np.testing.assert_allclose(M @ p, 0.5 * (p[sk.ek] + p[sk.el]), rtol=0, atol=1e-15)


def test_lemmas(p3d):
    """Lemma block-expansion and Lemma Ai-split (Eq. Ai-split-identity)."""
    *_, pc = p3d
    sk = pc.sk
    W, L, U, M, B, Z = oa.operators(sk)
    A = sk.A.toarray()
    Ahat = sp.block_diag(pc.A_loc).toarray()
    rng = np.random.default_rng(1)
    p = rng.standard_normal(sk.n)
    blocks = sum(p[a:b] @ A[a:b, a:b] @ p[a:b] for a, b in zip(sk.offsets[:-1], sk.offsets[1:]))
    uwl = p @ (U.T @ (W @ (L @ p)))
    assert np.isclose(p @ A @ p, blocks + 2 * uwl, rtol=1e-13)
    lwl = p @ (L.T @ (W @ (L @ p)))
    uwu = p @ (U.T @ (W @ (U @ p)))
    assert np.isclose(p @ Ahat @ p, blocks - lwl - uwu, rtol=1e-13)


def test_tildeA_identity(p2d, p3d):
    """Eq. (tildeA-identity) as matrices: A_hat + 4 M^T W M = A."""
    for *_, pc in (p2d, p3d):
        W, M, B, Z, Ahat, A = dense_ops(pc)
        np.testing.assert_allclose(Ahat + 4.0 * M.T @ W @ M, A, rtol=0,
                                   atol=1e-13 * np.abs(A).max())


def test_exact_rewrite(p3d):
    """Eq. (local-system-rewrite): A_hat p + B (M p) = A p for every p (no approximation)."""
    *_, pc = p3d
    W, M, B, Z, Ahat, A = dense_ops(pc)
    np.testing.assert_allclose(Ahat + B @ M, A, rtol=0, atol=1e-13 * np.abs(A).max())


def test_local_spd_and_weights(p3d):
    """A_i SPD when A is SPD and W < 0 (Sec. 3.3); diagonal of W negative (Eq. global-W)."""
    *_, pc = p3d
    assert (pc.sk.ea < 0).all()
    for Ai in pc.A_loc:
        np.linalg.cholesky(Ai.toarray())


def test_tpfa_remark_local_dirichlet():
    """Remark tpfa-local-dirichlet: for K = I on a uniform Cartesian grid, A_i equals the
    TPFA operator of the local Dirichlet problem on Omega_i (half-cell transmissibility
    2 at subdomain boundary faces), assembled here directly from the grid."""
    shape = (7, 6, 3)
    A, f = synth.tpfa_cartesian(np.ones(shape), bc_axis=0)
    part = op.partition(A, synth.even_part_sizes(A.shape[0], 5))
    sk = oa.skeleton(A, part)
    A_loc = oa.local_matrices(sk)
    nx, ny, nz = shape
    coords = np.array([(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)])
    for i in range(sk.m):
        cells = sk.perm[sk.offsets[i]:sk.offsets[i + 1]]        # original ids, ascending
        pos = {c: t for t, c in enumerate(cells)}
        Ad = np.zeros((len(cells), len(cells)))
        for t, c in enumerate(cells):
            x, y, z = coords[c]
            for ax in range(3):
                for d in (-1, 1):
                    q = [x, y, z]
                    q[ax] += d
                    if not (0 <= q[ax] < shape[ax]):
                        if ax == 0:                      # global Dirichlet face: T_b = 2
                            Ad[t, t] += 2.0
                        continue
                    nb = q[0] + nx * (q[1] + ny * q[2])
                    if nb in pos:                        # interior face: T = 1
                        Ad[t, t] += 1.0
                        Ad[t, pos[nb]] -= 1.0
                    else:                                # subdomain boundary: half cell
                        Ad[t, t] += 2.0
        np.testing.assert_allclose(A_loc[i].toarray(), Ad, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- preconditioner

def test_mbf_route_equals_dense_reduced(p2d, p3d):
    """Algorithm 2 through MBFs equals cal_M^{-1} r of Eq. (eq-m-reduced-p)."""
    rng = np.random.default_rng(2)
    for *_, pc in (p2d, p3d):
        r = rng.standard_normal(pc.sk.n)
        z = oa.apply(pc, r)
        zd = oa.apply_dense(pc, r)
        assert np.linalg.norm(z - zd) <= 1e-13 * np.linalg.norm(zd)


def test_interface_matrix_is_schur(p3d):
    """S equals -Z^T (W + W M A_hat^{-1} B) Z = Z^T S_lambda Z (Eq. k-schur) and is SPD."""
    *_, pc = p3d
    W, M, B, Z, Ahat, A = dense_ops(pc)
    S_lam = -(W + W @ M @ np.linalg.solve(Ahat, B))
    np.testing.assert_allclose(pc.S, Z.T @ S_lam @ Z, rtol=0, atol=1e-12 * np.abs(pc.S).max())
    assert np.linalg.eigvalsh(0.5 * (pc.S + pc.S.T)).min() > 0


def test_Q_spd_and_edge_form(p3d):
    """Thm. theorem:Q-psd: Q (Eq. Q-def) is SPD and satisfies Eq. (Q-edge-form)."""
    *_, pc = p3d
    W, M, B, Z, Ahat, A = dense_ops(pc)
    Q = np.block([[0.25 * Ahat, M.T @ W @ Z], [Z.T @ W @ M, -Z.T @ W @ Z]])
    np.testing.assert_array_equal(Q, Q.T)
    assert np.linalg.eigvalsh(Q).min() > 0
    rng = np.random.default_rng(3)
    p = rng.standard_normal(A.shape[0])
    eta = rng.standard_normal(Z.shape[1])
    v = np.concatenate([p, eta])
    lam = Z @ eta
    rhs = 0.25 * p @ A @ p - (lam - M @ p) @ W @ (lam - M @ p)
    assert np.isclose(v @ Q @ v, rhs, rtol=1e-12)


def test_single_subdomain_is_exact():
    """m = 1: A_hat = A, no interface, z = A^{-1} r; PCG converges in one iteration."""
    A, f, _ = small_problem(m=1)
    part = np.zeros(A.shape[0], dtype=np.int32)
    pc = oa.setup(A, part)
    r = np.random.default_rng(4).standard_normal(A.shape[0])
    x = np.linalg.solve(A.toarray(), r)
    np.testing.assert_allclose(oa.apply(pc, r), x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
    res = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-10)
    assert res.iterations == 1 and res.converged


def test_edge_mortar_recovers_A():
    """Lambda = R^E (Z = I): AlgMortar recovers the original system (Sec. 3.3), cal_M = A."""
    A, f, part = small_problem(shape=(6, 5, 2), m=3)
    pc = oa.setup(A, part, mortar="edge")
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    x = spla.spsolve(A.tocsc(), r)
    np.testing.assert_allclose(oa.apply(pc, r), x, rtol=0, atol=1e-11 * np.abs(x).max())
    np.testing.assert_allclose(oa.dense_reduced(pc), pc.sk.A.toarray(), atol=1e-12)


def test_chain_closed_form():
    """1D chain tridiag(-1, 2, -1): every E_ij holds one edge, so Lambda = R^E and z = A^{-1} r,
    with the closed-form Green's function (A^{-1})_ij = min(i,j)(N+1-max(i,j))/(N+1)."""
    N = 40
    A = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1], format="csr")
    part = op.partition(A, [10, 13, 9, 8])
    assert (np.diff(part) >= 0).all()                       # contiguous pieces
    pc = oa.setup(A, part)
    assert pc.sk.nLam == 3 and pc.sk.nE == 3
    i = np.arange(1, N + 1)
    Ainv = np.minimum.outer(i, i) * (N + 1 - np.maximum.outer(i, i)) / (N + 1)
    r = np.random.default_rng(6).standard_normal(N)
    np.testing.assert_allclose(oa.apply(pc, r), Ainv @ r, rtol=1e-12, atol=1e-12)


def test_interface_groups_all_edges_of_a_pair_by_hand():
    """Sec. 5.5: one psi per pair i~j, however many edges E_ij holds.  2 x 2 cells,
    unit transmissibilities, one unit Dirichlet face per cell (a_kk = 3), subdomains
    {0, 2} | {1, 3}: E_01 = {(0,1), (2,3)}.  By hand from the definitions:
      D_01 = diag(-1, -1), A_0 = A_1 = [[4, -1], [-1, 4]]             (Eq. A_i)
      G = B Z = (-2, -2, -2, -2), T = 2, Phi_i = -A_i^{-1} G_i = (2/3, 2/3)
      S_eta = T + G^T Phi / 4 = 2 - 16/12 = 2/3                      (Cor. cor-schur-eta)
    and for r = e_0: pbar = (4/15, 1/15 | 0, 0), b_eta = 1/6, eta = 1/4,
      z = pbar + Phi eta = (13/30, 5/30, 7/30, 5/30) in cells (0, 1, 2, 3),
    which differs from A^{-1} e_0 = (7/15, 1/5, 1/5, 2/15): the coarse space is one
    function, not one per edge.  A per-edge (or mis-grouped) Z fails every line."""
    A = sp.csr_matrix(np.array([[3., -1, -1, 0], [-1, 3, 0, -1], [-1, 0, 3, -1], [0, -1, -1, 3]]))
    part = np.array([0, 1, 0, 1])
    pc = oa.setup(A, part)
    assert pc.sk.nE == 2 and pc.sk.nLam == 1
    np.testing.assert_allclose(pc.S, [[2.0 / 3.0]], rtol=0, atol=1e-15)
    z = oa.apply(pc, np.array([1.0, 0, 0, 0]))
    np.testing.assert_allclose(z, np.array([13, 5, 7, 5]) / 30.0, rtol=0, atol=1e-15)
    assert np.abs(z - np.array([7 / 15, 1 / 5, 1 / 5, 2 / 15])).max() > 1e-2
    pbar, b_eta, eta, _ = oa.apply_parts(pc, np.array([1.0, 0, 0, 0]))
    np.testing.assert_allclose(pbar, [4 / 15, 1 / 15, 0, 0], rtol=0, atol=1e-15)   # (0, 2 | 1, 3)
    np.testing.assert_allclose(b_eta, [1 / 6], rtol=0, atol=1e-15)
    np.testing.assert_allclose(eta, [0.25], rtol=0, atol=1e-15)
    # the per-edge space Lambda = R^E has two unknowns here and recovers A^{-1}
    pe = oa.setup(A, part, mortar="edge")
    assert pe.S.shape == (2, 2)
    np.testing.assert_allclose(oa.apply(pe, np.array([1.0, 0, 0, 0])), [7 / 15, 1 / 5, 1 / 5, 2 / 15], atol=1e-15)


def test_multi_edge_interface_is_not_exact():
    """2D grid split into two halves: the one interface holds many edges, N_Lambda = 1,
    and z = cal_M^{-1} r differs from A^{-1} r (whereas the per-edge space recovers it)."""
    A, f, _ = small_problem(shape=(8, 6, 1), m=2)
    part = (np.arange(A.shape[0]) % 8 >= 4).astype(np.int32)   # x < 4 | x >= 4
    pc = oa.setup(A, part)
    assert pc.sk.nLam == 1 and pc.sk.nE == 6
    r = np.random.default_rng(21).standard_normal(A.shape[0])
    x = spla.spsolve(A.tocsc(), r)
    assert np.linalg.norm(oa.apply(pc, r) - x) > 1e-3 * np.linalg.norm(x)
    np.testing.assert_allclose(oa.apply(oa.setup(A, part, mortar="edge"), r), x, atol=1e-11 * np.abs(x).max())


def test_apply_parts_is_algorithm_2(p2d, p3d):
    """The staged form used by the GPU stage tests: its z equals apply()'s, and its eta
    solves the interface system S eta = b_eta."""
    for *_, pc in (p2d, p3d):
        r = np.random.default_rng(22).standard_normal(pc.sk.n)
        pbar, b_eta, eta, z = oa.apply_parts(pc, r)
        np.testing.assert_allclose(z[pc.sk.iperm], oa.apply(pc, r), rtol=0, atol=1e-13 * np.abs(z).max())
        assert np.linalg.norm(pc.S @ eta - b_eta) <= 1e-12 * np.linalg.norm(b_eta)
        # pbar solves the local systems A_i pbar_i = r_i (Eq. def-pbar-local)
        f = r[pc.sk.perm]
        for i, Ai in enumerate(pc.A_loc):
            a, b = pc.sk.offsets[i], pc.sk.offsets[i + 1]
            assert np.linalg.norm(Ai @ pbar[a:b] - f[a:b]) <= 1e-12 * np.linalg.norm(f[a:b])


def test_restriction_from_residual(p2d, p3d):
    """Algorithm 2's interface right-hand side -1/4 G^T pbar equals 1/4 Phi^T r: the MBFs
    are Phi = -A_hat^{-1} G (Eq. def-phat-local) and A_hat is symmetric, so the interface
    right-hand side depends on r alone (pins the oracle's MBFs and restriction together)."""
    for pc, n in ((p2d[3], p2d[0].shape[0]), (p3d[3], p3d[0].shape[0])):
        r = np.random.default_rng(21).standard_normal(n)
        _, rhs, _, _ = oa.apply_parts(pc, r)
        f = r[pc.sk.perm]
        alt = np.zeros_like(rhs)
        for i in range(pc.sk.m):
            a, b = pc.sk.offsets[i], pc.sk.offsets[i + 1]
            if pc.I_loc[i].size:
                np.add.at(alt, pc.I_loc[i], pc.Phat[i].T @ f[a:b])
        np.testing.assert_allclose(0.25 * alt, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_symmetry(p3d):
    """Cor. cor-schur-p: cal_M symmetric -> |r1.M^-1 r2 - r2.M^-1 r1| <= 1e-12 relative."""
    *_, pc = p3d
    rng = np.random.default_rng(7)
    r1, r2 = rng.standard_normal((2, pc.sk.n))
    a, b = r1 @ oa.apply(pc, r2), r2 @ oa.apply(pc, r1)
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_spectral_bounds(p2d, p3d):
    """Prop. bound-eigenvalues: 1/(1+K_Lambda) <= theta(cal_M^{-1} A) <= 1, and
    Thm. error-propagation-bound: kappa <= 1 + 2 K_Lambda, with K_Lambda of Eq. (k-lambda)
    from the generalised eigenproblem 4 M^T (-W)(I - Pi) M v = K A v."""
    for *_, pc in (p2d, p3d):
        W, M, B, Z, Ahat, A = dense_ops(pc)
        Mm = oa.dense_reduced(pc)
        theta = np.sort(np.real(sla.eigvals(np.linalg.solve(Mm, A))))
        Pi = Z @ np.linalg.solve(Z.T @ W @ Z, Z.T @ W)
        I = np.eye(W.shape[0])
        Nmat = 4.0 * M.T @ (I - Pi).T @ (-W) @ (I - Pi) @ M
        Nmat = 0.5 * (Nmat + Nmat.T)
        K = sla.eigh(Nmat, A, eigvals_only=True).max()
        assert theta.max() <= 1 + 1e-10
        assert theta.min() >= 1.0 / (1.0 + K) - 1e-10
        assert theta.max() / theta.min() <= 1 + 2 * K + 1e-8
        # the lower bound is attained (K_Lambda is a maximum over p)
        assert np.isclose(theta.min(), 1.0 / (1.0 + K), rtol=1e-8)


def test_interface_residual_structure(p3d):
    """Sec. 5.4: after an exact AlgMortar solve the residual r - A cal_M^{-1} r vanishes at
    every cell not adjacent to the partition interface."""
    *_, pc = p3d
    sk = pc.sk
    A = sp.csr_matrix(sk.A)
    r = np.random.default_rng(8).standard_normal(sk.n)
    z = oa.apply(pc, r[sk.iperm])[sk.perm]                  # permuted ordering
    res = r - A @ z
    iface = np.zeros(sk.n, dtype=bool)
    iface[sk.ek] = True
    iface[sk.el] = True
    assert np.abs(res[~iface]).max() <= 1e-12 * np.abs(r).max()
    assert np.abs(res[iface]).max() > 1e-6


def test_pcg_matches_direct_solve(p2d):
    """PCG (x0 = 0, Euclidean stop) reaches the dense Cholesky solution to the tolerance."""
    A, f, part, pc = p2d
    x = sla.cho_solve(sla.cho_factor(A.toarray()), f)
    res = oa.pcg(A, f, lambda v: oa.apply(pc, v), 1e-10)
    assert res.converged and res.rel_residual <= 1e-10
    kappa = np.linalg.cond(A.toarray())
    assert np.linalg.norm(res.x - x) <= 1e-10 * kappa * np.linalg.norm(x)
    plain = oa.pcg(A, f, lambda v: v.copy(), 1e-10)
    assert res.iterations < plain.iterations


def test_pcg_c1_converges():
    """Config 1 (64x64, 16 parts) converges to 1e-8 with far fewer iterations than CG."""
    P = synth.config1()
    part = op.partition(P.A, P.part_sizes)
    pc = oa.setup(P.A, part)
    res = oa.pcg(P.A, P.f, lambda v: oa.apply(pc, v), 1e-8)
    assert res.converged and res.iterations < 80
    xs = spla.spsolve(P.A.tocsc(), P.f)
    assert np.linalg.norm(res.x - xs) <= 1e-6 * np.linalg.norm(xs)


# ------------------------------------------------------------------ partition

def test_csgraph_bfs_is_fifo_ascending():
    """The library BFS used by the partitioner equals a plain FIFO queue BFS."""
    from scipy.sparse import csgraph
    rng = np.random.default_rng(9)
    for trial in range(20):
        n = 60
        R = sp.random(n, n, density=0.05, random_state=trial, format="csr")
        G = op.adjacency(R + R.T + sp.identity(n))
        s = int(rng.integers(n))
        ref = op.bfs_plain(G.indptr, G.indices, s)
        got = csgraph.breadth_first_order(G, s, directed=True, return_predecessors=False)
        assert list(got) == ref


def test_partition_golden():
    with open(os.path.join(GOLDEN, "partition_small.json")) as fh:
        gold = json.load(fh)
    for key in ("path6", "grid3x3"):
        g = gold[key]
        n = g["n"]
        e = np.array(g["edges"])
        A = sp.csr_matrix((-np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
        A = A + A.T + sp.identity(n) * 4
        assert list(op.partition(A, g["sizes"])) == g["part"]


def test_partition_sizes_and_determinism():
    P = synth.config1()
    a = op.partition(P.A, P.part_sizes)
    b = op.partition(P.A, P.part_sizes)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(np.bincount(a), P.part_sizes)
    sizes = synth.uneven_part_sizes(P.n, 7, 300, 900, 3)
    c = op.partition(P.A, sizes)
    np.testing.assert_array_equal(np.bincount(c), sizes)


# ------------------------------------------------------------------ adjoint

def test_adjoint_vs_central_fd():
    """dL/dlnK by the adjoint equals central finite differences (h = 1e-6, dense solves)."""
    shape = (5, 4, 3)
    lnK = synth.gaussian_field(shape, 2.0, 1.0, 77)
    A, f, faces = synth.tpfa_from_lnK(lnK, kz_ratio=0.1, bc_axis=0)
    rng = np.random.default_rng(78)
    obs = rng.choice(A.shape[0], 12, replace=False)
    p_obs = rng.uniform(0, 1, 12)
    solve = lambda M, v: sla.cho_solve(sla.cho_factor(M.toarray()), v)
    L, g, p, lam = oadj.grad_lnK(A, f, faces, lnK.ravel(order="F"), obs, p_obs, solve)
    h = 1e-6
    flat = lnK.ravel(order="F")
    for k in rng.choice(flat.size, 15, replace=False):
        vals = []
        for s in (1, -1):
            q = flat.copy()
            q[k] += s * h
            Ah, fh, _ = synth.tpfa_from_lnK(q.reshape(shape, order="F"), kz_ratio=0.1, bc_axis=0)
            vals.append(oadj.misfit(solve(Ah, fh), obs, p_obs))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g).max(), 1e-12)
