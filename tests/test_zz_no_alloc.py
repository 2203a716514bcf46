"""The allocation-free interface solve (algmortar_interface_solve_noalloc) against the
interface solution the regular path returns (algmortar_apply_stages), through the C ABI.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.  It also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import partition as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_22905_b300 import build
    build.build()


@pytest.mark.parametrize("depth", [0, 2])
def test_interface_solve_noalloc_matches_regular_path(depth):
    from paper_2607_22905_b300 import binding as B
    from paper_2607_22905_b300.solver import AlgMortar
    lnK = synth.gaussian_field((23, 19, 15), 3.0, 2.0, 41)
    A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=1)
    sizes = synth.uneven_part_sizes(A.shape[0], 16, 150, 900, 41)
    am = AlgMortar(A, len(sizes), part_sizes=sizes, nd_depth=depth)
    r = np.random.default_rng(7).standard_normal(A.shape[0])
    _, beta, eta, _ = am.apply_stages(r)
    beta = beta.contiguous()
    scale = float(torch.linalg.norm(eta))
    for _ in range(2):                     # two calls in a row share the static scratch
        out = torch.full_like(eta, float("nan"))
        rc = B.lib().algmortar_interface_solve_noalloc(am._h, C.c_void_p(beta.data_ptr()),
                                                       C.c_void_p(out.data_ptr()))
        assert rc == 0, B.lib().algmortar_last_error().decode()
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(out - eta)) <= 1e-10 * scale


def test_interface_solve_noalloc_smaller_call_after_larger():
    """The static array keeps the previous call's contents: a call on a smaller interface
    system right after a larger one (a different handle on the same GPU) must read only
    what it wrote itself; then the larger one again."""
    from paper_2607_22905_b300 import binding as B
    from paper_2607_22905_b300.solver import AlgMortar
    handles = []
    for shape, m, seed in (((25, 21, 17), 40, 43), ((12, 11, 9), 5, 44)):
        lnK = synth.gaussian_field(shape, 3.0, 2.0, seed)
        A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1, bc_axis=1)
        am = AlgMortar(A, m, part_sizes=synth.even_part_sizes(A.shape[0], m), nd_depth=1)
        r = np.random.default_rng(seed).standard_normal(A.shape[0])
        _, beta, eta, _ = am.apply_stages(r)
        handles.append((am, beta.contiguous(), eta))
    assert handles[0][2].numel() > 4 * handles[1][2].numel()
    for am, beta, eta in (handles[0], handles[1], handles[0], handles[1]):
        out = torch.full_like(eta, float("nan"))
        rc = B.lib().algmortar_interface_solve_noalloc(am._h, C.c_void_p(beta.data_ptr()),
                                                       C.c_void_p(out.data_ptr()))
        assert rc == 0, B.lib().algmortar_last_error().decode()
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(out - eta)) <= 1e-10 * float(torch.linalg.norm(eta))
        assert float((out - eta).abs().max()) <= 1e-10 * float(eta.abs().max())
