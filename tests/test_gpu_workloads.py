"""GPU against the oracle on reduced copies of the extra workloads: the cross-shaped
kappa = 1e6 field (Sec. 7.1 workload shape) and the K^theta contrast sweep of config 3's
field (Sec. 7.3): the FP64 preconditioner element-wise, the FP64 PCG iteration count and
solution, and the BF16 solve."""
import numpy as np
import pytest

import synth
from oracle import algmortar as oa
from oracle import partition as op

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    return max(float(np.linalg.norm(d)) / max(float(np.linalg.norm(b)), 1e-300),
               float(d.max(initial=0.0)) / max(float(np.abs(b).max(initial=0.0)), 1e-300))


REDUCED = {
    "cross_24": lambda: synth.config_cross(24, part_cells=700),
    "c3_theta0.6": lambda: synth.config3_theta(0.6, ny=12, n_parts=61),
    "c3_theta1.4": lambda: synth.config3_theta(1.4, ny=12, n_parts=61),
}


@pytest.fixture(scope="module", params=sorted(REDUCED))
def case(request):
    P = REDUCED[request.param]()
    part = op.partition(P.A, P.part_sizes)
    return request.param, P, part, oa.setup(P.A, part)


def test_apply_matches_oracle(case):
    from paper_2607_22905_b300.solver import AlgMortar
    name, P, part, pc = case
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes)
    np.testing.assert_array_equal(am.partition(), part)
    r = np.random.default_rng(7).standard_normal(P.n)
    assert rel(am.apply(r).cpu().numpy(), oa.apply(pc, r)) <= 1e-10


def test_pcg_matches_oracle(case):
    from paper_2607_22905_b300.solver import AlgMortar
    name, P, part, pc = case
    ref = oa.pcg(P.A, P.f, lambda r: oa.apply(pc, r), tol=1e-8)
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, use_graph=True, check_every=4)
    x, st = am.solve(P.f, tol=1e-8)
    assert st["status"] == 0 and abs(st["iterations"] - ref.iterations) <= 1
    assert rel(x.cpu().numpy(), ref.x) <= 1e-6
    lo = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision="bf16", use_graph=True, check_every=4)
    xb, sb = lo.solve(P.f, tol=1e-8)
    assert sb["status"] == 0
    assert np.linalg.norm(P.f - P.A @ xb.cpu().numpy()) <= 1e-8 * np.linalg.norm(P.f) * (1 + 1e-6)
