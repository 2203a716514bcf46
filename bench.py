"""Benchmark: time to a 1e-8 relative residual for AlgMortar-PCG on one B300.

Workload (default): the 1.122M-cell layered channelised 3D TPFA Darcy system
(60 x 220 x 85, contrast ~2e7, kz/kx = 0.1, 1122 uneven subdomains of ~300-3000 cells),
synthetic and seeded (see synth.config3).

One timed step = one full time-to-solution on device-resident inputs:
    numeric part of Algorithm 1 (local factors, MBFs, interface system, from the CSR
    values already in HBM)  +  PCG (x0 = 0) to ||r|| <= 1e-8 ||b||.
The host-side symbolic setup (partition of G(A), permutation, tables) depends only on
the sparsity pattern, is shared by all variants and is reported separately.

Variants differ only in the precision of the local factors / MBF panels (FP64, FP32,
BF16 with FP32 accumulation); SpMV, CG recurrences, dot products, restriction and the
interface solve are FP64 in all of them.  `value` is the fastest mixed-precision
variant; the FP64 variant is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica of the workload (weak scaling,
no data-path collective); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time-to-1e-8 rel. residual & PCG iters (1.1M cells): mixed/batched vs FP64 AlgMortar; "
          "HBM GB/s")
TOL = 1e-8


def _source_rev(rel):
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


# revision of the local-solve kernel source: DRAM traffic taken by ncu on another revision
# is not reported
KERNEL_REVISION = _source_rev("paper_2607_22905_b300/csrc/kernels_local.cu")
LOCAL_KERNEL = "k_chain_solve_pairs (batched local triangular solves, tile rows in pairs)"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


FLOOR = os.path.join(ROOT, "tests", "golden", "factor_floor.json")


def factor_floor(config, part):
    """sum_i nnz(L_i) of Algorithm 1's local factors under a fill-reducing order (stored
    by tests/golden/make_factor_floor.py from the oracle's symbolic count) for this
    workload, if the stored partition is the one the handle uses."""
    import hashlib
    try:
        with open(FLOOR) as fh:
            d = json.load(fh).get(config)
    except Exception:
        return None
    sha = hashlib.sha1(np.ascontiguousarray(part, dtype=np.int32).tobytes()).hexdigest()
    return d if d and d.get("partition_sha1") == sha else None


def workload(name):
    import synth
    if name == "c3":
        return synth.config3(), "C3 3D TPFA 60x220x85 (1.122M cells) layered channelised, contrast ~2e7, " \
                                "kz/kx=0.1, 1122 uneven parts"
    if name == "c3s":
        return synth.config3(ny=110, n_parts=561), "C3-small 60x110x85 (561k cells), same field recipe, 561 parts " \
                                                   "(profiling-sized case)"
    if name == "c2":
        return synth.config2(), "C2 3D TPFA 128^3 (2.1M cells), lnK~N(0,9), 512 parts"
    if name == "c1":
        return synth.config1(), "C1 2D TPFA 64x64, 16 parts"
    raise SystemExit(f"unknown workload {name}")


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile(prefix="clk_", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.n0 = 0
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: wait for its first sample, so that the
            # samples taken after it (rows n0 onwards) all fall inside the timed region
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.p.poll() is None:
                self.f.flush()
                if os.path.getsize(self.f.name) > 0:
                    break
                time.sleep(0.02)
            with open(self.f.name) as fh:
                self.n0 = sum(1 for _ in fh)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.close()

    def summary(self):
        rows = []
        try:
            for ln in open(self.f.name):
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        os.unlink(self.f.name)
        if len(rows) > self.n0:
            rows = rows[self.n0:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), world
    return None, 0, 1


def max_over_ranks(value, dist, device="cpu"):
    """Replica runs (one independent copy of the workload per rank, no data-path
    collective): the step time of the job is the slowest rank's."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    from paper_2607_22905_b300 import binding as B
    from paper_2607_22905_b300 import build as _build
    from paper_2607_22905_b300.solver import AlgMortar

    dist, rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _build.build()
    dev = torch.device("cuda", local)
    P, wdesc = workload(args.config)
    n, nnz = P.n, P.A.nnz
    vals = torch.as_tensor(P.A.data, dtype=torch.float64, device=dev)
    b = torch.as_tensor(P.f, dtype=torch.float64, device=dev)
    peak, peak_kind = load_peaks()
    variants = [v for v in args.variants.split(",") if v]
    res = {}
    handles = {}
    t0 = time.perf_counter()
    for v in variants:
        prec, iface = parse_variant(v)
        am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, use_graph=True,
                       check_every=args.check_every, device=local, interface_solve=iface,
                       autotune=not args.no_autotune)
        handles[v] = am
    host_setup_ms = {k: v.info["setup_ms"]["partition_and_tables"] for k, v in handles.items()}

    def step(am):
        am.update_values(vals)
        x, st = am.solve(b, tol=TOL)
        return x, st

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    clocks_all = {}
    for prec in variants:
        am = handles[prec]
        for _ in range(args.warmup):
            step(am)
        l0 = am.info["kernel_launches"] if "kernel_launches" in am.info else 0
        info0 = B.Info()
        B.check(B.lib().algmortar_get_info(am._h, C.byref(info0)))
        barrier()
        with Clocks() as clk:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            its = []
            for _ in range(args.steps):
                x, st = step(am)
                its.append(st["iterations"])
            e1.record()
            barrier()
        info1 = B.Info()
        B.check(B.lib().algmortar_get_info(am._h, C.byref(info1)))
        ms = e0.elapsed_time(e1) / args.steps
        ms = max_over_ranks(ms, dist, dev)
        xr = x.cpu().numpy()
        true_rel = float(np.linalg.norm(P.f - P.A @ xr) / np.linalg.norm(P.f))
        stages = am.time_stages(args.stage_reps)
        info = am.info
        res[prec] = {"ms": ms, "iterations": int(np.median(its)), "rel_residual": true_rel,
                     "interface_solve": parse_variant(prec)[1],
                     "iface_iterations_per_apply": (round(st["iface_iterations"] / (st["iterations"] + 1), 2)
                                                    if parse_variant(prec)[1] == "inexact" else None),
                     "setup_ms": {k: round(v, 3) for k, v in info["setup_ms"].items()},
                     "stages_ms": {k: round(v, 5) for k, v in stages.items()},
                     "launches_per_step": (info1.kernel_launches - info0.kernel_launches) / args.steps,
                     "tuned": {"local_solve_variant": info1.tuned_ring, "local_job_order": info1.tuned_job_order,
                               "vector_ctas_per_sm": info1.tuned_vec_ctas},
                     "factor_bytes": info["factor_bytes"], "n_lambda": info["n_lambda"],
                     "x_host": xr}
        clocks_all[prec] = clk.summary()

    # e2e: the same step through the C ABI with HOST buffers (pinned), copies inside
    mixed = [v for v in variants if v != "fp64"] or variants
    best = min(mixed, key=lambda v: res[v]["ms"])
    am = handles[best]
    vh = torch.as_tensor(P.A.data, dtype=torch.float64).pin_memory()
    bh = torch.as_tensor(P.f, dtype=torch.float64).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    L = B.lib()
    st = B.Stats()

    def e2e_step():
        B.check(L.algmortar_update_values(am._h, C.cast(C.c_void_p(vh.data_ptr()), B._DP)))
        rc = L.algmortar_pcg_solve_host(am._h, C.cast(C.c_void_p(bh.data_ptr()), B._DP),
                                        C.cast(C.c_void_p(xh.data_ptr()), B._DP), TOL, C.byref(st))
        B.check(rc, "algmortar_pcg_solve_host")

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    t = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - t) * 1e3 / args.steps

    # roofline of the dominant kernel: the batched local triangular solves.  Algorithmic
    # bytes = 2 s sum_i nnz(L_i) (both sweeps read every factor entry once, s bytes per
    # entry, nnz under a fill-reducing order) + 16 N (right-hand side in, solution out);
    # the bytes of the stored factor streams are reported beside them.
    r = res[best]
    best_prec, best_iface = parse_variant(best)
    isz = {"fp64": 8, "fp32": 4, "bf16": 2}[best_prec]
    fl = factor_floor(args.config, handles[best].partition())
    local_ms = r["stages_ms"]["local_solve"]
    stored_bytes = r["factor_bytes"] + 24 * n
    alg_bytes = 2 * isz * fl["sum_nnz_L"] + 16 * n if fl else None
    achieved = (alg_bytes if fl else stored_bytes) / (local_ms * 1e-3) / 1e9
    spmv_bytes = 12 * nnz + 4 * (n + 1) + 16 * n          # values+cols, rowptr, p read, q write
    vec_bytes = 72 * n                                     # p = z + beta p; x, r updates
    stage_gbs = {"spmv": round(spmv_bytes / (r["stages_ms"]["spmv"] * 1e-3) / 1e9, 1),
                 "cg_vectors": round(vec_bytes / (r["stages_ms"]["cg_vectors"] * 1e-3) / 1e9, 1)}
    out = {
        "metric": METRIC,
        "value": round(r["ms"], 3),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(r["ms"], 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{best_prec}+f64" + ("+f32" if best_iface == "inexact" else ""),
        "data": "synthetic",
        "config": {"workload": wdesc, "n": n, "nnz": nnz, "n_parts": P.n_parts, "n_lambda": r["n_lambda"],
                   "tol": TOL, "variant": best, "step": "numeric setup (Algorithm 1) + PCG to tol",
                   "l2": "inputs larger than L2 (factor streams %.2f GB, matrix %.0f MB)"
                         % (r["factor_bytes"] / 1e9, (12 * nnz) / 1e6),
                   "host_symbolic_setup_ms": round(host_setup_ms[best], 1)},
        "iterations": r["iterations"],
        "variants": {k: {kk: vv for kk, vv in v.items() if kk != "x_host"} for k, v in res.items()},
        "roofline": {"bound": "hbm", "kernel": LOCAL_KERNEL,
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": None,
                     "algorithmic_bytes": int(alg_bytes) if fl else None,
                     "floor": ("2 s sum_i nnz(L_i) + 16 N; nnz(L_i) = %d (oracle symbolic count, multiple "
                               "minimum degree), s = %d" % (fl["sum_nnz_L"], isz)) if fl else
                              "no stored floor for this partition: stored factor bytes used",
                     "stored_bytes": int(stored_bytes),
                     "stored_gbs": round(stored_bytes / (local_ms * 1e-3) / 1e9, 1),
                     "launch_ms": round(local_ms, 5),
                     "stages_gbs": stage_gbs,
                     "stages_frac": {k: round(v / peak, 4) for k, v in stage_gbs.items()}},
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": int(8 * nnz + 8 * n),
                "d2h_bytes_per_step": int(8 * n)},
        "gpu_launches": int(r["launches_per_step"] * args.steps),
        "clocks": clocks_all.get(best),
    }
    tr = load_traffic(best_prec)
    if tr is not None:
        out["roofline"]["traffic"] = tr["bytes_per_launch"]
        out["roofline"]["traffic_source"] = tr["source"]
    if "fp64" in res:
        out["fp64_ms"] = round(res["fp64"]["ms"], 3)
        out["speedup_vs_fp64"] = round(res["fp64"]["ms"] / r["ms"], 3)
    if args.extras and rank == 0:
        out["smoothing"] = smoothing_runs(P, best, vals, b, args, local)
        out["multi_rhs"] = multi_rhs_run(best, args, local)
        out["configs"] = config_runs(args, local)
        out["workloads"] = workload_runs(args, local)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(P, res.get("fp64", r)["iterations"])
    if rank == 0:
        print(json.dumps(out))
    for am in handles.values():
        am.close()
    if dist:
        dist.destroy_process_group()


def parse_variant(v):
    """'bf16' -> ('bf16', 'exact'); 'bf16-inexact' -> ('bf16', 'inexact'): local-factor
    precision and interface solve of Algorithm 2."""
    prec, _, iface = v.partition("-")
    return prec, (iface or "exact")


def load_traffic(variant):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary (scaled
    to the full workload there), or None when no summary covers this variant's kernel."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as fh:
            d = json.load(fh)
        e = d.get(variant)
        return e if e and e.get("kernel_revision") == KERNEL_REVISION else None
    except Exception:
        return None


def smoothing_runs(P, prec, vals, b, args, local, nus=(1, 2)):
    """Sec. 5.4 block-Jacobi pre/post smoothing (nu steps each side) on the same workload:
    step time (numeric setup + PCG to tol) and iterations, 2 timed steps each."""
    import torch
    from paper_2607_22905_b300.solver import AlgMortar
    outs = {}
    for nu in nus:
        am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, use_graph=True,
                       check_every=args.check_every, device=local, smooth_steps=nu)
        for _ in range(2):
            am.update_values(vals)
            am.solve(b, tol=TOL)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            am.update_values(vals)
            x, st = am.solve(b, tol=TOL)
        e1.record()
        torch.cuda.synchronize()
        outs[f"nu{nu}"] = {"ms": round(e0.elapsed_time(e1) / 2, 3), "iterations": st["iterations"],
                           "rel_residual": st["rel_residual"]}
        am.close()
    return outs


def multi_rhs_run(prec, args, local, nrhs=64, nsingle=4):
    """Batched multi-RHS PCG on config 4 (500k cells, irregular faulted grid, 64 RHS):
    one solve_multi call over all columns vs single-RHS solves of the same columns."""
    import torch
    import synth
    from paper_2607_22905_b300.solver import AlgMortar
    P = synth.config4()
    Bm = torch.as_tensor(P.meta["rhs"][:, :nrhs], dtype=torch.float64, device=torch.device("cuda", local))
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, use_graph=True,
                   check_every=args.check_every, device=local)
    am.solve_multi(Bm[:, :8], tol=TOL)
    am.solve(Bm[:, 0], tol=TOL)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    X, stats = am.solve_multi(Bm, tol=TOL)
    e[1].record()
    its1 = []
    e[2].record()
    for j in range(nsingle):
        x, st = am.solve(Bm[:, j], tol=TOL)
        its1.append(st["iterations"])
    e[3].record()
    torch.cuda.synchronize()
    batched = e[0].elapsed_time(e[1])
    single = e[2].elapsed_time(e[3]) / nsingle
    am.close()
    its = [s["iterations"] for s in stats]
    return {"workload": "C4 100x100x50 faulted hexahedral stand-in (500k cells), %d RHS, %s factors" % (nrhs, prec),
            "batched_ms_per_rhs": round(batched / nrhs, 3), "single_ms_per_rhs": round(single, 3),
            "batch_speedup": round(single / (batched / nrhs), 3),
            "iterations_min_max": [int(min(its)), int(max(its))], "single_iterations": its1}


def workload_runs(args, local, steps=2):
    """The extra synthetic workloads, each timed as a step of the headline (numeric setup +
    PCG to 1e-8, mean of `steps` after one warm-up): the cross-shaped kappa = 1e6 field on
    96^3 cells (864 even parts) in FP64 and BF16, and the K^theta contrast sweep of config
    3's field, theta = 0.6 ... 1.4, BF16 factors."""
    import torch
    import synth
    from paper_2607_22905_b300.solver import AlgMortar
    dev = torch.device("cuda", local)

    def run(P, prec):
        b = torch.as_tensor(P.f, dtype=torch.float64, device=dev)
        vals = torch.as_tensor(P.A.data, dtype=torch.float64, device=dev)
        am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, use_graph=True,
                       check_every=args.check_every, device=local)

        def step():
            am.update_values(vals)
            return am.solve(b, tol=TOL)[1]

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            st = step()
        e1.record()
        torch.cuda.synchronize()
        am.close()
        return {"ms": round(e0.elapsed_time(e1) / steps, 3), "iterations": st["iterations"],
                "rel_residual": st["rel_residual"]}

    out = {}
    P = synth.config_cross(96)
    out["cross_96"] = {"workload": P.name, "n": int(P.n), "n_parts": int(P.n_parts),
                       **{prec: run(P, prec) for prec in ("fp64", "bf16")}}
    sweep = {}
    for th in (0.6, 0.8, 1.0, 1.2, 1.4):
        P = synth.config3_theta(th)
        sweep[f"{th:g}"] = {"contrast": P.meta["contrast"], **run(P, "bf16")}
    out["c3_theta_bf16"] = sweep
    return out


def config_runs(args, local, steps=2):
    """The other workloads, each timed as a step of the headline (numeric setup + PCG to
    1e-8 on device-resident inputs, mean of `steps` after one warm-up): C1 (also the
    device time of one PCG iteration), C2 and C4 (first right-hand side) in every factor
    precision, and C5's batch of 8 permeability samples (loss and adjoint gradient
    dL/d ln K of each)."""
    import torch
    import synth
    from paper_2607_22905_b300.solver import AlgMortar
    dev = torch.device("cuda", local)
    outs = {}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, r

    for name, maker, rhs in (("c1", synth.config1, None), ("c2", synth.config2, None),
                             ("c4", synth.config4, "rhs0")):
        P = maker()
        b = torch.as_tensor(P.meta["rhs"][:, 0] if rhs else P.f, dtype=torch.float64, device=dev)
        vals = torch.as_tensor(P.A.data, dtype=torch.float64, device=dev)
        rows = {}
        for prec in ("fp64", "fp32", "bf16"):
            am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, use_graph=True,
                           check_every=args.check_every, device=local)

            def step():
                am.update_values(vals)
                return am.solve(b, tol=TOL)[1]

            ms, st = timed(step)
            row = {"ms": round(ms, 3), "iterations": st["iterations"], "rel_residual": st["rel_residual"]}
            if name == "c1":
                row["us_per_iteration"] = round(1e3 * am.time_stages(args.stage_reps)["iteration"], 2)
            rows[prec] = row
            am.close()
        outs[name] = {"workload": P.name, "n": int(P.n), "n_parts": int(P.n_parts), **rows}

    from paper_2607_22905_b300.adjoint import AlgMortarTPFASolve
    n = 96
    shape = (n, n, n)
    lnKs = [synth.gaussian_field(shape, 6.0, 2.0, s) for s in range(50, 58)]
    A0, f0, _ = synth.tpfa_from_lnK(synth.gaussian_field(shape, 6.0, 2.0, 5999))
    am = AlgMortar(A0, A0.shape[0] // 1728, precision="bf16", use_graph=True, check_every=args.check_every,
                   device=local)
    p_ref, _ = am.solve(f0, tol=TOL)
    obs, p_obs = synth.observations(A0.shape[0], 200, 5001, p_ref.cpu().numpy())
    o = torch.as_tensor(obs, device=dev)
    po = torch.as_tensor(p_obs, device=dev)

    def assemble(t):
        Ah, fh, fc = synth.tpfa_from_lnK(t.cpu().numpy().reshape(shape, order="F"))
        tb, tbp = synth.tpfa_cell_bc(Ah.shape[0], fc)
        return torch.as_tensor(Ah.data, device=dev), fh, tb, tbp

    flats = [torch.tensor(l.ravel(order="F"), device=dev) for l in lnKs]

    def batch():
        for fl in flats:
            x = fl.clone().requires_grad_(True)
            p = AlgMortarTPFASolve.apply(x, am, assemble, TOL)
            ((p[o] - po) ** 2).sum().backward()

    ms, _ = timed(batch)
    am.close()
    outs["c5"] = {"workload": "C5 96^3 TPFA, ln K ~ N(0, 2^2), 8 samples: forward solve + adjoint solve + "
                              "dL/d ln K each (host assembly of A(ln K) included), bf16 factors",
                  "n": int(A0.shape[0]), "ms_per_batch_of_8": round(ms, 3)}
    return outs


def cpu_baseline(P, iters, n_iter_sample=8):
    """The FP64 CPU oracle, as it stands, on the host cores, on a bounded sample of the
    workload: its Algorithm 1 setup on the full workload, then the first n_iter_sample
    iterations of its own PCG (oracle.algmortar.pcg_iterations) timed; the time to
    solution is the setup plus iters times the mean iteration (iters = the FP64 GPU
    count, which the parity tests hold within one of the oracle's)."""
    from oracle import algmortar as oa
    from oracle import partition as op
    t0 = time.perf_counter()
    part = op.partition(P.A, P.part_sizes)
    t_part = time.perf_counter() - t0
    t0 = time.perf_counter()
    pc = oa.setup(P.A, part)
    t_setup = time.perf_counter() - t0
    gen = oa.pcg_iterations(P.A, P.f, lambda v: oa.apply(pc, v), TOL)
    t0 = time.perf_counter()
    done = 0
    for _ in range(n_iter_sample):
        try:
            next(gen)
            done += 1
        except StopIteration:
            break
    t_it = (time.perf_counter() - t0) / max(done, 1)
    value = t_setup + iters * t_it
    return {"value": round(value * 1e3, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle Algorithm 1 setup on the full workload ({t_setup:.1f} s) + the first {done} "
                      f"iterations of the oracle's PCG ({t_it * 1e3:.0f} ms each, initial preconditioner "
                      f"application included) scaled to {iters} iterations (the FP64 GPU count); host "
                      f"partition ({t_part:.1f} s) excluded as on the GPU side"}


def run_reference(args, est_iters=200):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores (rank 0 only),
    ONE whole time to solution measured: the host partition untimed (as on the GPU
    side); the first warm-up step times Algorithm 1 (oracle.algmortar.setup); the K
    timed steps then run the oracle's own PCG (oracle.algmortar.pcg_iterations) ceil(200
    / K) iterations each until it stops (steps left after the stop run iterations of a
    second solve, not counted).  value = setup + the time of the first solve's
    iterations; ms_per_step = the mean timed step.  If the K steps end before the solve
    stops, it is run to the end after them and still counted."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import math
    from oracle import algmortar as oa
    from oracle import partition as op
    P, wdesc = workload(args.config)
    part = op.partition(P.A, P.part_sizes)
    t0 = time.perf_counter()
    pc = oa.setup(P.A, part)
    t_setup = time.perf_counter() - t0
    precond = lambda v: oa.apply(pc, v)
    for _ in range(max(0, args.warmup - 1)):
        precond(P.f)
    per_step = max(1, math.ceil(est_iters / max(args.steps, 1)))
    gen = oa.pcg_iterations(P.A, P.f, precond, TOL)
    result, t_solve, extra = None, 0.0, None
    step_s = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            if result is None:
                ta = time.perf_counter()
                try:
                    next(gen)
                except StopIteration as stop:
                    result = stop.value
                t_solve += time.perf_counter() - ta
                if result is not None:
                    break
            else:                               # keep the step's work: a second solve
                if extra is None:
                    extra = oa.pcg_iterations(P.A, P.f, precond, TOL)
                try:
                    next(extra)
                except StopIteration:
                    extra = None
        step_s.append(time.perf_counter() - t0)
    while result is None:                       # K steps were not enough: finish it
        ta = time.perf_counter()
        try:
            next(gen)
        except StopIteration as stop:
            result = stop.value
        t_solve += time.perf_counter() - ta
    value = 1e3 * (t_setup + t_solve)
    ms_step = 1e3 * sum(step_s) / max(len(step_s), 1)
    cb = {"value": round(value, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"one whole oracle time to solution: Algorithm 1 setup ({t_setup * 1e3:.0f} ms) + its PCG to "
                    f"{TOL:g} ({result.iterations} iterations, {t_solve * 1e3:.0f} ms, true rel. residual "
                    f"{result.rel_residual:.2e}), spread over the timed steps ({per_step} iterations a step); "
                    f"host partition excluded as on the GPU side"}
    out = {"metric": METRIC, "value": cb["value"], "unit": "ms", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": wdesc, "n": P.n, "nnz": P.A.nnz, "n_parts": P.n_parts, "tol": TOL},
           "iterations": result.iterations,
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_apply(args):
    """One setup and one application of the preconditioner (kernel profiling target)."""
    import torch
    from paper_2607_22905_b300.solver import AlgMortar
    P, wdesc = workload(args.config)
    prec, iface = parse_variant(args.variants.split(",")[0])
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, interface_solve=iface)
    r = torch.as_tensor(np.random.default_rng(0).standard_normal(P.n), device="cuda")
    z = am.apply(r)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "apply", "workload": wdesc, "variant": prec, "info": am.info,
                      "z_norm": float(z.norm())}))
    am.close()


def run_solve(args):
    """One setup and one PCG solve to the tolerance on the stream path (profiling target
    for the per-iteration kernels)."""
    import torch
    from paper_2607_22905_b300.solver import AlgMortar
    P, wdesc = workload(args.config)
    prec, iface = parse_variant(args.variants.split(",")[0])
    am = AlgMortar(P.A, P.n_parts, part_sizes=P.part_sizes, precision=prec, interface_solve=iface)
    x, st = am.solve(torch.as_tensor(P.f, device="cuda"), tol=TOL)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "solve", "workload": wdesc, "variant": prec, "stats": st}))
    am.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3")
    ap.add_argument("--variants", default="fp64,fp32,bf16,bf16-inexact")
    ap.add_argument("--check-every", type=int, default=8)
    ap.add_argument("--stage-reps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="built-in launch variants instead of the autotuner's (setup-time) choice")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the smoothing and multi-RHS side measurements")
    ap.add_argument("--mode", default="bench", choices=["bench", "apply", "solve"],
                    help="apply / solve: set up the first variant and run one preconditioner "
                         "application / one PCG solve (kernel profiling targets), no timing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "apply":
        run_apply(args)
    elif args.mode == "solve":
        run_solve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
