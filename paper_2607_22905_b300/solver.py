"""PyTorch-facing wrapper of the AlgMortar-PCG library.

PyTorch supplies device memory and the stream; the work runs in libalgmortar's kernels.
There is no CPU fallback: without a CUDA device or without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import binding as B


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


class AlgMortar:
    """AlgMortar preconditioner + PCG for an SPD scipy CSR matrix A (original ordering).

    precision: "fp64" | "fp32" | "bf16" for the local factors/solves and MBF panels.
    part_sizes: optional target sizes of the n_parts subdomains (sum = N).
    parts: optional labels replacing the built-in partitioner.
    interface_solve: "exact" (FP64) or "inexact" (block-Jacobi PCG in FP32 to iface_rtol,
    blocks of interfaces (i, j) with equal i // iface_block_parts; flexible outer CG).
    autotune: time the hot kernels' launch variants on this problem during setup.
    seed: with part_sizes None, nonzero draws uneven target sizes (algmortar_part_sizes).
    stage_times: per-stage device times of the last PCG iteration in the solve stats.
    """

    def __init__(self, A, n_parts, precision="fp64", part_sizes=None, parts=None, use_graph=False,
                 check_every=1, max_it=10000, diag_scale=True, device=0, verbose=False, stream=None,
                 nd_depth=-1, flexible=False, smooth_steps=0, interface_solve="exact", iface_rtol=1e-2,
                 iface_block_parts=1, iface_max_it=200, autotune=False, seed=0, stage_times=False):
        if not torch.cuda.is_available():
            raise RuntimeError("AlgMortar needs a CUDA device")
        L = B.lib()
        self.n = int(A.shape[0])
        self.device = torch.device("cuda", device)
        o = B.default_opts()
        o.precision = B.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.diag_scale = 1 if diag_scale else 0
        o.max_it = int(max_it)
        o.use_graph = 1 if use_graph else 0
        o.check_every = int(check_every)
        o.verbose = 1 if verbose else 0
        o.device = int(device)
        o.nd_depth = int(nd_depth)
        o.flexible = 1 if flexible else 0
        o.smooth_steps = int(smooth_steps)
        o.interface_solve = {"exact": B.IFACE_EXACT, "inexact": B.IFACE_INEXACT}[interface_solve]
        o.iface_rtol = float(iface_rtol)
        o.iface_block_parts = int(iface_block_parts)
        o.iface_max_it = int(iface_max_it)
        o.autotune = 1 if autotune else 0
        o.seed = int(seed)
        o.stage_times = 1 if stage_times else 0
        self._sizes = None
        if part_sizes is not None:
            self._sizes = np.ascontiguousarray(part_sizes, dtype=np.int32)
            o.part_sizes = self._sizes.ctypes.data_as(B._IP)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        o.stream = C.c_void_p(stream.cuda_stream) if stream.cuda_stream else None
        self._stream = stream
        csr = B.csr_struct(A)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            if parts is not None:
                p = np.ascontiguousarray(parts, dtype=np.int32)
                B.check(L.algmortar_setup_with_parts(C.byref(csr), p.ctypes.data_as(B._IP), int(n_parts),
                                                     C.byref(o), C.byref(h)), "algmortar_setup_with_parts")
            else:
                B.check(L.algmortar_setup(C.byref(csr), int(n_parts), C.byref(o), C.byref(h)),
                        "algmortar_setup")
        self._h = h
        self.values_token = object()
        info = B.Info()
        B.check(L.algmortar_get_info(h, C.byref(info)))
        self.info = info.as_dict()

    # -------------------------------------------------------------- helpers
    def _vec(self, v):
        v = torch.as_tensor(v, dtype=torch.float64, device=self.device)
        return v.contiguous()

    def close(self):
        if getattr(self, "_h", None):
            B.lib().algmortar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def apply(self, r):
        """z = cal_M^{-1} r (Algorithm 2)."""
        r = self._vec(r)
        z = torch.empty_like(r)
        B.check(B.lib().algmortar_apply(self._h, _ptr(r), _ptr(z)), "algmortar_apply")
        return z

    def apply_stages(self, r):
        """(pbar, b_eta, eta, z) of Algorithm 2 in the internal ordering."""
        r = self._vec(r)
        nl = max(self.info["n_lambda"], 1)
        pbar = torch.empty_like(r)
        z = torch.empty_like(r)
        beta = torch.empty(nl, dtype=torch.float64, device=self.device)
        eta = torch.empty_like(beta)
        B.check(B.lib().algmortar_apply_stages(self._h, _ptr(r), _ptr(pbar), _ptr(beta), _ptr(eta), _ptr(z)))
        nl = self.info["n_lambda"]
        return pbar, beta[:nl], eta[:nl], z

    def solve(self, b, tol=1e-8, raise_on_fail=True, history=0):
        """PCG with x0 = 0 to ||r|| <= tol ||b||; returns (x, stats dict).  history > 0:
        stats["history"] holds ||r_k|| / ||b|| for the first `history` iterates."""
        b = self._vec(b)
        x = torch.empty_like(b)
        st = B.Stats()
        hbuf = None
        if history > 0:
            hbuf = (C.c_double * int(history))()
            st.history = C.cast(hbuf, C.POINTER(C.c_double))
            st.history_len = int(history)
        rc = B.lib().algmortar_pcg_solve(self._h, _ptr(b), _ptr(x), float(tol), C.byref(st))
        if raise_on_fail and rc != B.OK:
            raise B.AlgMortarError(rc, "algmortar_pcg_solve")
        d = st.as_dict()
        del hbuf
        return x, d

    def solve_host(self, b, tol=1e-8):
        """PCG with HOST numpy b -> host x (copies inside the call)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        st = B.Stats()
        rc = B.lib().algmortar_pcg_solve_host(self._h, b.ctypes.data_as(B._DP), x.ctypes.data_as(B._DP),
                                              float(tol), C.byref(st))
        if rc != B.OK:
            raise B.AlgMortarError(rc, "algmortar_pcg_solve_host")
        return x, st.as_dict()

    def solve_multi(self, Bm, tol=1e-8, raise_on_fail=True):
        """Independent PCG solves for the columns of an N x k matrix, batched: each
        iteration's kernels cover all columns of a batch in one launch."""
        Bm = torch.as_tensor(Bm, dtype=torch.float64, device=self.device)
        Bt = Bm.t().contiguous()                      # k x N row-major == N x k column-major
        Xt = torch.empty_like(Bt)
        k = Bt.shape[0]
        st = (B.Stats * k)()
        rc = B.lib().algmortar_pcg_solve_multi(self._h, _ptr(Bt), _ptr(Xt), k, self.n, float(tol), st)
        if rc != B.OK and (raise_on_fail or rc not in (B.NO_CONVERGENCE, B.BREAKDOWN)):
            raise B.AlgMortarError(rc, "algmortar_pcg_solve_multi")
        return Xt.t(), [s.as_dict() for s in st]

    def update_values(self, values):
        """New CSR values (same pattern, original CSR order): numpy -> host path,
        CUDA tensor -> device path.  Re-runs the numeric part of Algorithm 1."""
        if isinstance(values, torch.Tensor) and values.is_cuda:
            v = values.to(torch.float64).contiguous()
            B.check(B.lib().algmortar_update_values_device(self._h, _ptr(v)), "algmortar_update_values_device")
        else:
            v = np.ascontiguousarray(values, dtype=np.float64)
            B.check(B.lib().algmortar_update_values(self._h, v.ctypes.data_as(B._DP)), "algmortar_update_values")
        self.values_token = object()
        info = B.Info()
        B.check(B.lib().algmortar_get_info(self._h, C.byref(info)))
        self.info = info.as_dict()

    def tpfa_grad_lnK(self, K, tb, tbp, p, lam):
        """dL/d ln K for TPFA values (see algmortar_tpfa_grad_lnK); device tensors."""
        K, tb, tbp, p, lam = (self._vec(v) for v in (K, tb, tbp, p, lam))
        out = torch.empty_like(p)
        B.check(B.lib().algmortar_tpfa_grad_lnK(self._h, _ptr(K), _ptr(tb), _ptr(tbp), _ptr(p), _ptr(lam),
                                                _ptr(out)), "algmortar_tpfa_grad_lnK")
        return out

    STAGES = ("spmv", "cg_vectors", "local_solve", "restrict", "coarse", "prolong", "iteration")

    def time_stages(self, reps=20):
        """Average device ms per PCG-iteration stage (CUDA events on the handle's stream)."""
        out = (C.c_double * 8)()
        B.check(B.lib().algmortar_time_stages(self._h, int(reps), out), "algmortar_time_stages")
        return dict(zip(self.STAGES, list(out)[:7]))

    def get_info(self):
        """Fresh algmortar_info (device-side counters such as iface_last_iterations)."""
        info = B.Info()
        B.check(B.lib().algmortar_get_info(self._h, C.byref(info)))
        return info.as_dict()

    def partition(self):
        out = np.empty(self.n, dtype=np.int32)
        B.check(B.lib().algmortar_get_partition(self._h, out.ctypes.data_as(B._IP)))
        return out

    def permutation(self):
        out = np.empty(self.n, dtype=np.int32)
        B.check(B.lib().algmortar_get_permutation(self._h, out.ctypes.data_as(B._IP)))
        return out

    def interfaces(self):
        nl = self.info["n_lambda"]
        out = np.empty(2 * max(nl, 1), dtype=np.int32)
        B.check(B.lib().algmortar_get_interfaces(self._h, out.ctypes.data_as(B._IP)))
        return out[:2 * nl].reshape(nl, 2)
