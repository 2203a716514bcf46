"""Seeded synthetic inputs: TPFA Darcy pressure matrices and partition size targets.

This module produces the *inputs* of the AlgMortar preconditioner (an SPD matrix A,
a right-hand side f, and the list of subdomain sizes handed to the graph partitioner).
It holds none of the method's arithmetic: no partitioning, no local operators, no
interface system, no Krylov iteration.  Both the CUDA path and the CPU oracle consume
what it returns.

The matrices are two-point flux approximations (TPFA) of -div(K grad p) = 0 on unit
cells, the discretisation the paper uses in its numerical experiments (Sec. 7):

* interior face between cells k and l: T_kl = 2 K_k K_l / (K_k + K_l) (harmonic mean),
  scaled by the face's area/distance factor;
* Dirichlet face of cell k: T_b = 2 K_k (half-cell), contributing T_b to a_kk and
  T_b * p_bc to f_k;
* a_kk = sum of the cell's face transmissibilities, a_kl = -T_kl.

All off-diagonals are therefore <= 0, and A is SPD as soon as one Dirichlet face exists
in every connected component.

Random numbers: numpy's PCG64 (`numpy.random.default_rng(seed)`) for fields, and
SplitMix64 (Steele, Lea & Flood 2014) for the integer size weights of uneven partitions.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem", "gaussian_field", "tpfa_cartesian", "config1", "config2", "config3",
    "config4", "config5", "tpfa_from_lnK", "even_part_sizes", "uneven_part_sizes", "splitmix64",
    "PAPER_WORKLOADS", "EXTRA_WORKLOADS", "cross_field", "config_cross", "config3_theta",
]


@dataclasses.dataclass
class Problem:
    """One synthetic linear system A p = f in CSR form (original cell ordering)."""

    name: str
    A: sp.csr_matrix            # N x N, FP64, full symmetric pattern, sorted columns
    f: np.ndarray               # length N, FP64
    shape: tuple                # grid shape (nx, ny, nz)
    n_parts: int                # number of subdomains the workload asks for
    part_sizes: np.ndarray      # int32 target sizes, sum == N
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]


# ----------------------------------------------------------------------------------
# random fields
# ----------------------------------------------------------------------------------

def gaussian_field(shape, corr_len: float, sigma: float, seed: int) -> np.ndarray:
    """Stationary Gaussian field with covariance ~ sigma^2 exp(-r^2 / (2 l^2)).

    White noise from PCG64(seed) is convolved (periodic FFT) with a Gaussian kernel of
    standard deviation l / sqrt(2) (the self-convolution of that kernel has standard
    deviation l), then standardised to sample mean 0 / std 1 and scaled by sigma.
    Returned array has shape `shape` indexed [x, y, z].
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    s = corr_len / np.sqrt(2.0)
    spec = np.fft.fftn(w)
    for ax, n in enumerate(shape):
        if n == 1:
            continue
        k = np.fft.fftfreq(n) * 2.0 * np.pi
        g = np.exp(-0.5 * (k * s) ** 2)
        bshape = [1] * len(shape)
        bshape[ax] = n
        spec = spec * g.reshape(bshape)
    field = np.real(np.fft.ifftn(spec))
    field = (field - field.mean()) / max(field.std(), 1e-300)
    return sigma * field


# ----------------------------------------------------------------------------------
# TPFA assembly on a Cartesian grid
# ----------------------------------------------------------------------------------

def cell_index(shape):
    nx, ny, nz = shape
    return np.arange(nx * ny * nz, dtype=np.int64).reshape((nz, ny, nx)).transpose(2, 1, 0)


def tpfa_faces(K: np.ndarray, kz_ratio: float = 1.0, face_scale=None):
    """Interior faces (k, l, T_kl, axis) of a Cartesian grid with cell permeability K.

    Cells are numbered x fastest: idx = x + nx*(y + ny*z).  `face_scale`, if given, is a
    dict axis -> array of per-face area/distance factors (shape of the face set).
    """
    nx, ny, nz = K.shape
    idx = cell_index(K.shape)
    ks, ls, ts, axes = [], [], [], []
    for axis in range(3):
        if K.shape[axis] == 1:
            continue
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[axis] = slice(0, K.shape[axis] - 1)
        sl_b[axis] = slice(1, K.shape[axis])
        Ka, Kb = K[tuple(sl_a)], K[tuple(sl_b)]
        if axis == 2:
            Ka, Kb = Ka * kz_ratio, Kb * kz_ratio
        T = 2.0 * Ka * Kb / (Ka + Kb)
        if face_scale is not None and axis in face_scale:
            T = T * face_scale[axis]
        ks.append(idx[tuple(sl_a)].ravel(order="F"))
        ls.append(idx[tuple(sl_b)].ravel(order="F"))
        ts.append(T.ravel(order="F"))
        axes.append(np.full(T.size, axis, dtype=np.int8))
    return (np.concatenate(ks), np.concatenate(ls), np.concatenate(ts), np.concatenate(axes))


def dirichlet_faces(K: np.ndarray, axis: int, p_lo: float, p_hi: float, kz_ratio=1.0):
    """Half-cell Dirichlet faces on the low/high ends of `axis`: (cell, T_b, p_bc)."""
    idx = cell_index(K.shape)
    Kx = K * (kz_ratio if axis == 2 else 1.0)
    cells, tb, pbc = [], [], []
    for end, pv in ((0, p_lo), (K.shape[axis] - 1, p_hi)):
        sl = [slice(None)] * 3
        sl[axis] = slice(end, end + 1)
        cells.append(idx[tuple(sl)].ravel(order="F"))
        tb.append(2.0 * Kx[tuple(sl)].ravel(order="F"))
        pbc.append(np.full(cells[-1].size, pv))
    return np.concatenate(cells), np.concatenate(tb), np.concatenate(pbc)


def assemble(n, k, l, T, bc_cells, bc_T, bc_p):
    """A = sum_faces T (e_k - e_l)(e_k - e_l)^T + sum_bc T_b e_k e_k^T; f = sum_bc T_b p_bc e_k."""
    rows = np.concatenate([k, l, k, l])
    cols = np.concatenate([l, k, k, l])
    vals = np.concatenate([-T, -T, T, T])
    rows = np.concatenate([rows, bc_cells])
    cols = np.concatenate([cols, bc_cells])
    vals = np.concatenate([vals, bc_T])
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A.eliminate_zeros()
    f = np.zeros(n)
    np.add.at(f, bc_cells, bc_T * bc_p)
    return A.astype(np.float64), f


def tpfa_cartesian(K: np.ndarray, kz_ratio=1.0, bc_axis=0, p_lo=1.0, p_hi=0.0, face_scale=None):
    """TPFA matrix and RHS for cell permeability K (shape nx, ny, nz), Dirichlet on the
    two ends of `bc_axis`, no-flow elsewhere."""
    n = K.size
    k, l, T, _ = tpfa_faces(K, kz_ratio, face_scale)
    c, tb, pb = dirichlet_faces(K, bc_axis, p_lo, p_hi, kz_ratio)
    return assemble(n, k, l, T, c, tb, pb)


# ----------------------------------------------------------------------------------
# partition size targets
# ----------------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser applied to state x + golden gamma (Steele et al. 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def even_part_sizes(n: int, m: int) -> np.ndarray:
    """m sizes differing by at most one, larger ones first, summing to n."""
    base, extra = divmod(n, m)
    s = np.full(m, base, dtype=np.int64)
    s[:extra] += 1
    return s.astype(np.int32)


def uneven_part_sizes(n: int, m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """m skewed sizes summing exactly to n, roughly within [lo, hi].

    Weight w_j = lo + (hi - lo) * u1 * u2 with u1, u2 uniform from SplitMix64(seed, j):
    a right-skewed spread (mean lo + (hi-lo)/4).  Sizes are the integer differences of
    floor(n * C_j / W) over the cumulative weights C_j, so they sum to n exactly.
    """
    K = 1 << 20
    w = np.empty(m, dtype=object)
    for j in range(m):
        a = splitmix64((seed << 32) ^ (2 * j)) % K
        b = splitmix64((seed << 32) ^ (2 * j + 1)) % K
        w[j] = lo * K * K + (hi - lo) * a * b
    C = np.cumsum(w)
    W = int(C[-1])
    cuts = [0] + [(n * int(c)) // W for c in C]
    s = np.diff(np.array(cuts, dtype=np.int64))
    assert s.sum() == n and (s > 0).all()
    return s.astype(np.int32)


# ----------------------------------------------------------------------------------
# the five workloads (the paper's SPE10/SPE11/cross-field inputs are not available;
# these synthetic stand-ins reproduce their shape, size and contrast)
# ----------------------------------------------------------------------------------

def config1(seed: int = 1) -> Problem:
    """2D 64x64, ln K ~ N(0,1), corr. length 4, Dirichlet p=1 left / p=0 right, 16 parts."""
    shape = (64, 64, 1)
    lnK = gaussian_field(shape, 4.0, 1.0, seed)
    A, f = tpfa_cartesian(np.exp(lnK), bc_axis=0)
    return Problem("c1_2d_64x64", A, f, shape, 16, even_part_sizes(A.shape[0], 16),
                   {"lnK": lnK})


def config2(seed: int = 2, n: int = 128, n_parts: int = 512) -> Problem:
    """3D n^3, ln K ~ N(0, 3^2), corr. length 8, kz/kx = 0.1, 512 parts of ~4096."""
    shape = (n, n, n)
    lnK = gaussian_field(shape, 8.0, 3.0, seed)
    A, f = tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=0)
    return Problem(f"c2_3d_{n}cube", A, f, shape, n_parts,
                   even_part_sizes(A.shape[0], n_parts), {})


def channel_field(shape, n_top: int, seed: int):
    """Layered channelised permeability (mD) indexed [x, y, z], z = 0 at the top.

    Top `n_top` layers: smooth log-normal (sigma 1.5, corr. length 6) clipped to
    [1e-3, 2e4].  Remaining layers: binary sinuous channels along y of width 2-6 cells,
    2e4 mD inside, 1e-3 mD background (contrast 2e7), about a quarter of the volume.
    """
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    K = np.empty(shape)
    top = gaussian_field((nx, ny, n_top), 6.0, 1.5, seed + 1000)
    K[:, :, :n_top] = np.clip(np.exp(np.log(20.0) + top), 1e-3, 2e4)
    y = np.arange(ny)
    xg = np.arange(nx)[:, None]
    bottom = np.zeros((nx, ny, nz - n_top), dtype=bool)
    z = 0
    while z < nz - n_top:
        thick = int(rng.integers(2, 5))
        layer = np.zeros((nx, ny), dtype=bool)
        n_ch = int(rng.integers(3, 6))
        for _ in range(n_ch):
            x0 = rng.uniform(0, nx)
            amp = rng.uniform(3, 12)
            lam = rng.uniform(40, 120)
            ph = rng.uniform(0, 2 * np.pi)
            width = rng.uniform(2, 6)
            xc = x0 + amp * np.sin(2 * np.pi * y / lam + ph)
            layer |= np.abs(xg - xc[None, :]) <= width / 2
        bottom[:, :, z:z + thick] = layer[:, :, None]
        z += thick
    K[:, :, n_top:] = np.where(bottom, 2e4, 1e-3)
    return K


def config3(seed: int = 3, n_parts: int = 1122, ny: int = 220) -> Problem:
    """3D 60x220x85 (1.122M cells): 35 smooth top layers over 50 channelised layers,
    contrast ~2e7, kz/kx = 0.1, Dirichlet on the y ends, uneven parts of ~300-3000.
    `ny` < 220 gives a shorter copy of the same field (profiling-sized case)."""
    shape = (60, ny, 85)
    K = channel_field(shape, 35, seed)
    A, f = tpfa_cartesian(K, kz_ratio=0.1, bc_axis=1)
    sizes = uneven_part_sizes(A.shape[0], n_parts, 300, 3000, seed)
    return Problem(f"c3_3d_60x{ny}x85_channels", A, f, shape, n_parts, sizes,
                   {"channel_fraction": float((K[:, :, 35:] > 1).mean())})


def config4(seed: int = 4, shape=(100, 100, 50), n_parts: int = 500, nrhs: int = 64) -> Problem:
    """Irregular faulted hexahedral stand-in: 500k cells, 8-12 off-diagonals, 64 RHS.

    Geometry enters through per-connection area/distance factors:
    * node perturbations up to +-30% of the cell size scale every face factor in
      [0.4, 1.9] and add in-plane diagonal (x+-1, y+-1) connections with 5-15% of the
      face transmissibility (the non-orthogonal part of an irregular hexahedron);
    * 10% of cells are pinched to 1e-3 of their thickness (their horizontal faces
      shrink by 1e-4, their vertical half-distances by the same factor);
    * 5 vertical faults (x = const planes) with throws of 1-5 layers replace the
      straight x-face by two non-neighbour connections to the shifted column (overlap
      fractions 0.6 / 0.4).
    Every off-diagonal is -T <= 0; the transmissibility contrast exceeds 1e8.
    """
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    K = np.exp(gaussian_field(shape, 5.0, 0.5, seed + 400))
    n = nx * ny * nz
    idx = cell_index(shape)
    thick = np.where(rng.random(shape) < 0.10, 1e-3, 1.0)
    faults = np.sort(rng.choice(np.arange(5, nx - 5), size=5, replace=False))
    throws = rng.integers(1, 6, size=5)
    ks, ls, ts = [], [], []

    def hm(a, b):
        return 1.0 / (0.5 / a + 0.5 / b)

    for axis in range(3):
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[axis] = slice(0, shape[axis] - 1)
        sl_b[axis] = slice(1, shape[axis])
        Ka, Kb = K[tuple(sl_a)], K[tuple(sl_b)]
        ta, tb_ = thick[tuple(sl_a)], thick[tuple(sl_b)]
        if axis == 2:
            T = 1.0 / (0.5 * ta / (0.1 * Ka) + 0.5 * tb_ / (0.1 * Kb))
        else:
            T = np.minimum(ta, tb_) * hm(Ka, Kb)
        T = T * rng.uniform(0.4, 1.9, size=T.shape)
        kk, ll = idx[tuple(sl_a)], idx[tuple(sl_b)]
        mask = np.ones(T.shape, dtype=bool)
        if axis == 0:
            for fx, th in zip(faults, throws):
                mask[fx, :, :] = False
                for dz, frac in ((int(th), 0.6), (int(th) + 1, 0.4)):
                    zs = np.arange(nz - dz)
                    Kf, Kg = K[fx][:, zs], K[fx + 1][:, zs + dz]
                    hf = np.minimum(thick[fx][:, zs], thick[fx + 1][:, zs + dz])
                    ks.append(idx[fx][:, zs].ravel())
                    ls.append(idx[fx + 1][:, zs + dz].ravel())
                    ts.append((frac * hf * hm(Kf, Kg)).ravel())
        ks.append(kk[mask]); ls.append(ll[mask]); ts.append(T[mask])
    for dy in (1, -1):
        ya = slice(0, ny - 1) if dy == 1 else slice(1, ny)
        yb = slice(1, ny) if dy == 1 else slice(0, ny - 1)
        a = (slice(0, nx - 1), ya, slice(None))
        b = (slice(1, nx), yb, slice(None))
        T = np.minimum(thick[a], thick[b]) * hm(K[a], K[b]) * rng.uniform(0.05, 0.15, size=K[a].shape)
        ks.append(idx[a].ravel()); ls.append(idx[b].ravel()); ts.append(T.ravel())
    k = np.concatenate(ks); l = np.concatenate(ls); T = np.concatenate(ts)
    c, tbv, pb = dirichlet_faces(K * thick, 0, 1.0, 0.0)
    A, f = assemble(n, np.minimum(k, l), np.maximum(k, l), T, c, tbv, pb)
    rhs = np.stack([np.random.default_rng(4000 + j).standard_normal(n) for j in range(nrhs)], 1)
    sizes = uneven_part_sizes(n, n_parts, 300, 3000, seed)
    return Problem("c4_3d_100x100x50_faulted", A, f, shape, n_parts, sizes,
                   {"rhs": rhs, "faults": faults.tolist(), "throws": throws.tolist()})


def tpfa_cell_bc(n, faces):
    """Per-cell sums of the Dirichlet half-faces: tb_k = sum_b T_b, tbp_k = sum_b T_b p_bc."""
    tb = np.zeros(n)
    tbp = np.zeros(n)
    np.add.at(tb, faces["bc_cell"], faces["bc_T"])
    np.add.at(tbp, faces["bc_cell"], faces["bc_T"] * faces["bc_p"])
    return tb, tbp


def observations(n, n_obs, seed, p_ref, noise=0.01):
    """Seeded observation cells (without replacement) and noisy observed pressures."""
    rng = np.random.default_rng(seed)
    obs = np.sort(rng.choice(n, n_obs, replace=False))
    return obs, p_ref[obs] + noise * rng.standard_normal(n_obs)


def tpfa_from_lnK(lnK: np.ndarray, kz_ratio=1.0, bc_axis=0, p_lo=1.0, p_hi=0.0):
    """TPFA system for log-permeability lnK plus the face data the gradient needs.

    Returns (A, f, faces) with faces = dict(k, l, T, bc_cell, bc_T, bc_p): interior
    faces T_kl = 2 K_k K_l / (K_k + K_l) and Dirichlet half-faces T_b = 2 K_k.
    """
    K = np.exp(lnK)
    k, l, T, _ = tpfa_faces(K, kz_ratio)
    c, tb, pb = dirichlet_faces(K, bc_axis, p_lo, p_hi, kz_ratio)
    A, f = assemble(K.size, k, l, T, c, tb, pb)
    return A, f, dict(k=k, l=l, T=T, bc_cell=c, bc_T=tb, bc_p=pb)


def config5(seed: int = 50, n: int = 96, n_parts: Optional[int] = None) -> Problem:
    """3D n^3 TPFA, ln K ~ N(0, 2^2), corr. length 6 (one sample of the gradient batch)."""
    shape = (n, n, n)
    lnK = gaussian_field(shape, 6.0, 2.0, seed)
    A, f = tpfa_cartesian(np.exp(lnK), bc_axis=0)
    N = A.shape[0]
    m = n_parts if n_parts is not None else max(1, N // 1728)
    return Problem(f"c5_3d_{n}cube_s{seed}", A, f, shape, m, even_part_sizes(N, m),
                   {"lnK": lnK})


def cross_field(n: int, motif: int = 8, kappa: float = 1e6) -> np.ndarray:
    """Cross-shaped high-contrast permeability on an n^3 grid (Sec. 7.1 workload shape).

    In every motif^3 block, cell (i, j, k) (block-local indices) has K = kappa when at
    least two of i, j, k lie in the block's central band {motif/2 - 1, motif/2}: three
    orthogonal bars of 2 x 2 cells through the block centre.  Periodic replication joins
    the bars of neighbouring blocks into channels along every axis; K = 1 elsewhere.
    (The paper gives the motif as a figure only; this is the reading used here.)
    """
    idx = np.arange(n) % motif
    band = (idx == motif // 2 - 1) | (idx == motif // 2)
    bi, bj, bk = np.meshgrid(band, band, band, indexing="ij")
    cnt = bi.astype(int) + bj.astype(int) + bk.astype(int)
    return np.where(cnt >= 2, kappa, 1.0)


def config_cross(n: int = 96, motif: int = 8, kappa: float = 1e6, part_cells: int = 1024) -> Problem:
    """Unit cube, n^3 cells, cross-shaped field with contrast kappa; p = 0 on y = 0 and
    p = 1 on y = 1, no flow elsewhere, zero source; even parts of ~part_cells cells."""
    shape = (n, n, n)
    K = cross_field(n, motif, kappa)
    A, f = tpfa_cartesian(K, kz_ratio=1.0, bc_axis=1, p_lo=0.0, p_hi=1.0)
    m = max(1, A.shape[0] // part_cells)
    return Problem(f"cross_{n}cube_kappa{kappa:.0e}", A, f, shape, m, even_part_sizes(A.shape[0], m),
                   {"high_fraction": float((K > 1).mean()), "kappa": kappa, "motif": motif})


def config3_theta(theta: float, seed: int = 3, n_parts: int = 1122, ny: int = 220) -> Problem:
    """Contrast sweep (Sec. 7.3): config 3's field K replaced by K^theta, so a contrast c
    becomes c^theta; everything else as config 3."""
    shape = (60, ny, 85)
    K = channel_field(shape, 35, seed) ** float(theta)
    A, f = tpfa_cartesian(K, kz_ratio=0.1, bc_axis=1)
    sizes = uneven_part_sizes(A.shape[0], n_parts, 300, 3000, seed)
    return Problem(f"c3_theta{theta:g}", A, f, shape, n_parts, sizes,
                   {"theta": float(theta), "contrast": float(K.max() / K.min())})


PAPER_WORKLOADS = {
    "c1": config1, "c2": config2, "c3": config3, "c4": config4, "c5": config5,
}
EXTRA_WORKLOADS = {"cross": config_cross, "c3_theta": config3_theta}
