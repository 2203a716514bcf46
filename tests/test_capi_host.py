"""CPU-only checks of the C ABI: the library loads, exports every declared entry point,
and its host-side steps (validation, partition) behave -- no kernel runs here."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import partition as op
from paper_2607_22905_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2607_22905_b300 import build
    build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "algmortar.h")).read()
    decl = r"^\s*(?:int|void|const char\s*\*)\s*(algmortar_[A-Za-z0-9_]+)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


def test_exports_every_declared_symbol():
    L = B.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(B.SIGNATURES)


def test_library_resolves_every_symbol_at_load():
    """dlopen with RTLD_NOW: a missing template instantiation or kernel symbol fails here
    instead of at its first call on the GPU."""
    import ctypes
    ctypes.CDLL(B.LIB_PATH, mode=ctypes.RTLD_GLOBAL | os.RTLD_NOW)


def test_strerror_and_defaults():
    L = B.lib()
    for s in range(10):
        assert L.algmortar_strerror(s)
    o = B.default_opts()
    assert o.precision == B.FP64 and o.diag_scale == 1 and o.max_it == 10000
    assert o.interface_solve == B.IFACE_EXACT and o.iface_block_parts == 1 and o.iface_max_it == 200
    assert o.iface_rtol == 1e-2 and o.autotune == 0 and o.seed == 0 and o.stage_times == 0


@pytest.mark.parametrize("cfg", ["config1"])
def test_partition_bit_identical_to_oracle(cfg):
    P = getattr(synth, cfg)()
    np.testing.assert_array_equal(B.partition(P.A, P.n_parts, P.part_sizes), op.partition(P.A, P.part_sizes))


@pytest.mark.parametrize("n,m,seed", [(1122000, 1122, 3), (500000, 500, 4), (5000, 7, 11), (640, 64, 1)])
def test_uneven_part_sizes_match_the_generator(n, m, seed):
    """The library's seeded size draw (opts.seed) equals the workload generator's rule with
    lo = 3n/(10m), hi = 3n/m -- 300..3000 for the 1.122M-cell and 500k-cell cases."""
    out = np.empty(m, dtype=np.int32)
    B.check(B.lib().algmortar_part_sizes(n, m, seed, out.ctypes.data_as(B._IP)))
    ref = synth.uneven_part_sizes(n, m, 3 * n // (10 * m), 3 * n // m, seed)
    np.testing.assert_array_equal(out, ref)
    assert out.sum() == n


def test_uneven_part_sizes_rejects_bad_arguments():
    out = np.empty(4, dtype=np.int32)
    assert B.lib().algmortar_part_sizes(3, 4, 1, out.ctypes.data_as(B._IP)) == B.INVALID_ARG
    assert B.lib().algmortar_part_sizes(10, 0, 1, out.ctypes.data_as(B._IP)) == B.INVALID_ARG


def test_partition_uneven_and_3d():
    lnK = synth.gaussian_field((14, 11, 9), 3.0, 2.0, 21)
    A, f = synth.tpfa_cartesian(np.exp(lnK), kz_ratio=0.1)
    sizes = synth.uneven_part_sizes(A.shape[0], 9, 60, 400, 5)
    np.testing.assert_array_equal(B.partition(A, 9, sizes), op.partition(A, sizes))
    np.testing.assert_array_equal(B.partition(A, 7), op.partition(A, synth.even_part_sizes(A.shape[0], 7)))


def test_partition_disconnected_graph():
    # two disjoint 1D chains plus an isolated node: BFS must continue into each component
    n = 23
    rows, cols = [], []
    for a, b in [(0, 10), (10, 22)]:
        for i in range(a, b - 1):
            rows += [i, i + 1]
            cols += [i + 1, i]
    A = sp.csr_matrix((-np.ones(len(rows)), (rows, cols)), shape=(n, n)) + 3 * sp.identity(n)
    A = sp.csr_matrix(A)
    A.sort_indices()
    for sizes in ([5, 6, 12], [1, 1, 21], [11, 12]):
        np.testing.assert_array_equal(B.partition(A, len(sizes), sizes), op.partition(A, sizes))


def test_golden_partitions_through_library():
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "partition_small.json")))
    for key in ("path6", "grid3x3"):
        g = gold[key]
        e = np.array(g["edges"])
        n = g["n"]
        A = sp.csr_matrix((-np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(n, n))
        A = sp.csr_matrix(A + A.T + 4 * sp.identity(n))
        A.sort_indices()
        assert list(B.partition(A, len(g["sizes"]), g["sizes"])) == g["part"]


def _setup_status(A, n_parts):
    import ctypes as C
    s = B.csr_struct(A)
    h = C.c_void_p()
    o = B.default_opts()
    rc = B.lib().algmortar_setup(C.byref(s), n_parts, C.byref(o), C.byref(h))
    assert not h.value
    return rc, B.lib().algmortar_last_error().decode()


def test_setup_rejects_bad_inputs_on_host():
    """Validation runs on the host before any device work: error codes, no trap."""
    A = synth.config1().A.copy()
    # non-symmetric value
    B2 = A.copy().tolil()
    B2[0, 1] = B2[0, 1] * 1.5
    assert _setup_status(sp.csr_matrix(B2), 4)[0] == B.NOT_SYMMETRIC
    # positive coupling between subdomains (W not negative definite)
    B3 = A.copy().tolil()
    part = op.partition(A, synth.even_part_sizes(A.shape[0], 4))
    k = next(i for i in range(A.shape[0]) if part[i] == 0 and any(part[j] != 0 for j in A[i].indices))
    l = next(j for j in A[k].indices if part[j] != 0)
    B3[k, l] = 0.5
    B3[l, k] = 0.5
    rc, msg = _setup_status(sp.csr_matrix(B3), 4)
    assert rc == B.INTERFACE_SIGN, msg
    # NaN value
    B4 = A.copy()
    B4.data[5] = np.nan
    assert _setup_status(B4, 4)[0] == B.INVALID_ARG
    # more parts than rows
    assert _setup_status(A, A.shape[0] + 1)[0] == B.INVALID_ARG
    # missing diagonal
    B5 = A.copy().tolil()
    B5[3, 3] = 0.0
    B5 = sp.csr_matrix(B5)
    B5.eliminate_zeros()
    assert _setup_status(B5, 4)[0] == B.INVALID_ARG
