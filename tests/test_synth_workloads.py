"""CPU checks of the extra synthetic workloads: the cross-shaped high-contrast field
(Sec. 7.1 workload shape) and the K^theta contrast sweep on config 3's field (Sec. 7.3)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import algmortar as oa
from oracle import partition as op


def test_cross_motif_by_hand():
    K = synth.cross_field(8, 8, 1e6)
    # three orthogonal 2x2 bars through the centre of the 8^3 motif: 3*(2*2*6) + 2*2*2 cells
    assert int((K > 1).sum()) == 3 * 24 + 8
    assert K[3, 3, 0] == 1e6 and K[0, 4, 3] == 1e6 and K[4, 0, 4] == 1e6
    assert K[3, 0, 0] == 1.0 and K[0, 0, 0] == 1.0 and K[7, 7, 7] == 1.0
    assert set(np.unique(K)) == {1.0, 1e6}


def test_cross_is_periodic_and_connected_along_y():
    K = synth.cross_field(24, 8, 1e6)
    assert np.array_equal(K[:8, :8, :8], K[8:16, 16:24, :8])
    # a high-permeability channel spans y from face to face
    assert (K[3, :, 3] > 1).all() and (K[4, :, 4] > 1).all()


def test_cross_problem_is_an_spd_m_matrix():
    P = synth.config_cross(16)
    A = P.A
    assert P.n == 16 ** 3 and P.part_sizes.sum() == P.n
    assert abs(A - A.T).max() == 0.0
    off = A - sp.diags(A.diagonal())
    assert off.max() <= 0.0
    # Dirichlet on y = 0 (p = 0) and y = 1 (p = 1): the source is nonzero only next to y = 1
    f = P.f.reshape(16, 16, 16)
    assert np.all(f[:, :-1, :] == 0.0) and np.all(f[:, -1, :] > 0.0)
    assert np.linalg.eigvalsh(A.toarray()).min() > 0.0


def test_theta_one_is_config3_and_contrast_scales():
    a = synth.config3(ny=24)
    b = synth.config3_theta(1.0, ny=24)
    assert (a.A != b.A).nnz == 0 and np.array_equal(a.f, b.f)
    c1 = synth.config3_theta(1.0, ny=24).meta["contrast"]
    for th in (0.6, 1.4):
        c = synth.config3_theta(th, ny=24).meta["contrast"]
        assert np.isclose(np.log(c), th * np.log(c1), rtol=1e-12)


def test_oracle_pcg_on_a_reduced_cross():
    P = synth.config_cross(16)
    part = op.partition(P.A, P.part_sizes)
    pc = oa.setup(P.A, part)
    res = oa.pcg(P.A, P.f, lambda r: oa.apply(pc, r), tol=1e-8)
    assert res.converged and res.rel_residual <= 1e-8
