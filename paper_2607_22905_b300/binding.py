"""ctypes marshalling for libalgmortar.so (C ABI in include/algmortar.h).

Argument marshalling only: every step of the solver runs in the library's CUDA kernels.
The library is loaded on first use from this directory and a missing build raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libalgmortar.so")

OK, INVALID_ARG, NOT_SYMMETRIC, INTERFACE_SIGN, NOT_SPD, NO_CONVERGENCE, BREAKDOWN, CUDA, OOM, TOO_LARGE = range(10)
FP64, FP32, BF16 = 0, 1, 2
IFACE_EXACT, IFACE_INEXACT = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16}


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.POINTER(C.c_int32)),
                ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("diag_scale", C.c_int32), ("max_it", C.c_int32),
                ("use_graph", C.c_int32), ("check_every", C.c_int32), ("flexible", C.c_int32),
                ("verbose", C.c_int32), ("device", C.c_int32), ("part_sizes", C.POINTER(C.c_int32)),
                ("stream", C.c_void_p), ("nd_depth", C.c_int32), ("autotune", C.c_int32),
                ("interface_solve", C.c_int32), ("smooth_steps", C.c_int32), ("iface_block_parts", C.c_int32),
                ("iface_max_it", C.c_int32), ("stage_times", C.c_int32), ("iface_rtol", C.c_double),
                ("seed", C.c_uint64)]


STAGE_NAMES = ("spmv", "cg_vectors", "local_solve", "restrict", "coarse", "prolong")


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("recursive_residual", C.c_double), ("solve_ms", C.c_double), ("host_ms", C.c_double),
                ("stage_ms", C.c_double * 6), ("iface_iterations", C.c_int64),
                ("history", C.POINTER(C.c_double)), ("history_len", C.c_int32), ("history_count", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("stage_ms", "history", "history_len")}
        d["stage_ms"] = dict(zip(STAGE_NAMES, list(self.stage_ms)))
        if self.history and self.history_count > 0:
            d["history"] = [self.history[i] for i in range(self.history_count)]
        return d


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_parts", C.c_int32), ("n_lambda", C.c_int32), ("max_part", C.c_int32),
                ("min_part", C.c_int32), ("precision", C.c_int32), ("n_interface_edges", C.c_int64),
                ("factor_entries", C.c_int64), ("factor_bytes", C.c_int64), ("phi_entries", C.c_int64),
                ("setup_ms", C.c_double * 8), ("kernel_launches", C.c_int64), ("interface_solve", C.c_int32),
                ("iface_blocks", C.c_int32), ("iface_cluster", C.c_int32), ("iface_staged", C.c_int32),
                ("iface_last_iterations", C.c_int32), ("tuned_ring", C.c_int32), ("tuned_vec_ctas", C.c_int32),
                ("tuned_job_order", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "setup_ms"}
        names = ["partition_and_tables", "upload", "local_factor", "mbf", "interface_assemble",
                 "interface_factor_inverse", "interface_factor", "total"]
        d["setup_ms"] = dict(zip(names, list(self.setup_ms)))
        return d


_P = C.c_void_p
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
SIGNATURES = {
    "algmortar_default_opts": (None, [C.POINTER(Opts)]),
    "algmortar_partition": (C.c_int, [C.POINTER(Csr), C.c_int32, _IP, _IP]),
    "algmortar_part_sizes": (C.c_int, [C.c_int64, C.c_int32, C.c_uint64, _IP]),
    "algmortar_setup": (C.c_int, [C.POINTER(Csr), C.c_int32, C.POINTER(Opts), C.POINTER(_P)]),
    "algmortar_setup_with_parts": (C.c_int, [C.POINTER(Csr), _IP, C.c_int32, C.POINTER(Opts), C.POINTER(_P)]),
    "algmortar_apply": (C.c_int, [_P, _P, _P]),
    "algmortar_apply_stages": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "algmortar_pcg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.POINTER(Stats)]),
    "algmortar_pcg_solve_host": (C.c_int, [_P, _DP, _DP, C.c_double, C.POINTER(Stats)]),
    "algmortar_pcg_solve_multi": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int64, C.c_double, C.POINTER(Stats)]),
    "algmortar_update_values": (C.c_int, [_P, _DP]),
    "algmortar_update_values_device": (C.c_int, [_P, _P]),
    "algmortar_tpfa_grad_lnK": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "algmortar_interface_solve_noalloc": (C.c_int, [_P, _P, _P]),
    "algmortar_get_partition": (C.c_int, [_P, _IP]),
    "algmortar_get_permutation": (C.c_int, [_P, _IP]),
    "algmortar_get_interfaces": (C.c_int, [_P, _IP]),
    "algmortar_get_info": (C.c_int, [_P, C.POINTER(Info)]),
    "algmortar_time_stages": (C.c_int, [_P, C.c_int32, _DP]),
    "algmortar_destroy": (None, [_P]),
    "algmortar_strerror": (C.c_char_p, [C.c_int]),
    "algmortar_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libalgmortar.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_22905_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class AlgMortarError(RuntimeError):
    def __init__(self, status, where=""):
        L = lib()
        self.status = status
        msg = L.algmortar_strerror(status).decode()
        detail = L.algmortar_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})" if where else f"{msg} ({detail})")


def check(status, where=""):
    if status != OK:
        raise AlgMortarError(status, where)
    return status


def csr_struct(A):
    """Csr struct viewing scipy CSR arrays (keeps references alive on the struct)."""
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    col = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    s = Csr(A.shape[0], len(val), rowptr.ctypes.data_as(_IP), col.ctypes.data_as(_IP), val.ctypes.data_as(_DP))
    s._keep = (rowptr, col, val)
    return s


def default_opts():
    o = Opts()
    lib().algmortar_default_opts(C.byref(o))
    return o


def partition(A, n_parts, part_sizes=None):
    """Host-only partition of G(A) by the library (no GPU needed)."""
    s = csr_struct(A)
    out = np.empty(A.shape[0], dtype=np.int32)
    sizes = None
    if part_sizes is not None:
        sizes = np.ascontiguousarray(part_sizes, dtype=np.int32)
    check(lib().algmortar_partition(C.byref(s), int(n_parts),
                                    sizes.ctypes.data_as(_IP) if sizes is not None else None,
                                    out.ctypes.data_as(_IP)), "algmortar_partition")
    return out
