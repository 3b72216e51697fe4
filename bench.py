#!/usr/bin/env python3
"""Benchmark: circulant-preconditioned voxel VIE solves on GB300.

One step = one complete solve of the workload through the libvie C ABI:
set the permittivity (material operator M), build the block-diagonal
Chan-Olkin preconditioner (Chan eigenvalues, block assembly, reduction, FP64
LU, complex-FP32 inverse), and run complex-FP32 GMRES(50) inside FP64
iterative refinement to the FP64 relative residual 1e-9.

Default workload: the 1024x16x8 long straight silicon wire (h = 0.025 um,
lambda = 1.55 um, 10% absorbers).  N > 1 GPUs run independent replicas (one
solve per rank per step, no collective on the data path).

Printed JSON: value = solves/s over all ranks (device time, inputs resident),
e2e = the same through vie_solve_host with host buffers (copies timed),
fp64_gpu = the plain FP64 GPU solver on the same problem, roofline = the
dominant kernel of the solve against the measured peak, cpu_baseline = the
CPU oracle on a bounded sample scaled to one solve.

--impl reference times the CPU oracle alone (bounded samples, host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VIE solves/s at 1e-6 rel. err (mixed vs FP64 GPU); matvec HBM GB/s; p50/p99 ms"
UNIT = "solves/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_PEAK_TFLOPS = 1.196      # DFMA probe on this machine's GB300 (152 SMs at 2.07 GHz)
FP32_PEAK_TFLOPS = 69.94      # FFMA probe, same run


def workload(name):
    from paper_1903_07884_gb300 import inputs
    if name == "long_straight":
        return inputs.workload_long_straight(), "long_straight_1024x16x8"
    if name == "small_straight":
        return inputs.workload_small_straight(), "small_straight_64x8x4"
    if name == "bragg":
        return inputs.workload_bragg(), "bragg_4096x24x8_2boxes"
    if name == "coupler":
        return inputs.workload_coupler(), "coupler_2048x48x8_2boxes"
    if name == "coupler_batch":      # the batch's first wavelength (the batch itself runs in run_batch)
        return inputs.workload_coupler(wavelength=1.50), "coupler_2048x48x8_2boxes_lambda1.50"
    raise SystemExit(f"unknown workload {name}")


def aggregate_ms(ms_local: float, world: int, dist=None, device=None) -> float:
    """Max over ranks of the per-step time (replicas: every rank solves its own
    copy of the workload; the job is as slow as its slowest rank)."""
    if world <= 1 or dist is None:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def solves_per_s(ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank finishes one solve per step."""
    return world * 1000.0 / ms_max


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work per launch of the kernels that can dominate a solve
# ---------------------------------------------------------------------------
def algorithmic(kernel: str, p, plan_meta: dict):
    """(kind, amount per launch) or None, for the complex-FP32 kernels of the
    solve (8 bytes per complex value).  Byte counts are the minimum each
    kernel must move; the matvec intermediate T is the yz-transformed field
    [3][Py][Pz][nx] of the three-pass scheme."""
    nx, ny, nz = p.nx, p.ny, p.nz
    N = nx * ny * nz
    n3 = 3 * N
    L, Py, Pz = 2 * _smooth(nx), 2 * _smooth(ny), 2 * _smooth(nz)
    T = 3 * nx * Py * Pz
    oct_ = 6 * (L // 2 + 1) * (Py // 2 + 1) * (Pz // 2 + 1)
    c = 8
    jbar = plan_meta.get("mean_j", 25.0)           # mean Arnoldi step index j over the launches
    if kernel == "mv_yz_fwd_c64":
        return "hbm", c * (n3 + T)
    if kernel == "mv_x_c64":
        return "hbm", c * (2 * T + oct_)
    if kernel == "mv_yz_inv_c64":
        return "hbm", c * (T + n3 + N + n3)
    k = plan_meta.get("plans_per_launch", 1)     # the Arnoldi kernels cover every plan of a batch per launch
    if kernel == "arnoldi_dot_c64":       # reads w, u_j and V_0..V_{j-1}
        return "hbm", k * c * (jbar + 2) * n3
    if kernel == "arnoldi_update_c64":    # reads the same, writes q_j and w''
        return "hbm", k * c * (jbar + 4) * n3
    if kernel == "block_gemv_c64":
        m, nh = plan_meta["m"], plan_meta["nhalf"]
        return "hbm", c * nh * m * m
    if kernel == "rep_gemm_tc":
        m, nd = plan_meta["m"], plan_meta["ndisc"]
        return "tensor", 8.0 * nd * m * m              # nd x m x m complex multiply-adds
    if kernel in ("lu_update", "lu_update_c64"):
        # trailing updates A22 -= L21 U12 of the blocked LU (panels of 16): 8 real flops per
        # complex multiply-add, averaged over the panel steps (one launch per step and box);
        # complex FP64 for the FP64 preconditioner, complex FP32 for the mixed one
        m, nblk = plan_meta["m"], plan_meta["nblk"]
        steps = [(k0, min(16, m - k0)) for k0 in range(0, m, 16) if m - k0 - min(16, m - k0) > 0]
        flops = sum(8.0 * nb * (m - k0 - nb) ** 2 for k0, nb in steps)
        return "alu", nblk * flops / len(steps)
    return None


# DRAM bytes (read + write) per launch from one ncu --set full capture of the
# same kernel versions on the 1024x16x8 wire: per basis column read for the
# Arnoldi reduction (325.7 MB at step j = 100, j + 2 = 102 columns), per
# launch for the others.  Cleared whenever a kernel changes.
TRAFFIC = {
    "long_straight_1024x16x8": {
        "arnoldi_dot_c64": ("per_column", 325.70e6 / 102),
        "mv_x_c64": ("per_launch", 20.23e6),
        "block_gemv_c64": ("per_launch", 132.30e6),
    }
}


MV_KERNELS = ("mv_yz_fwd_c64", "mv_x_c64", "mv_yz_inv_c64")


def matvec_summary(table: dict, p, hbm_gbs: float):
    """Complex-FP32 matvec bandwidth from the per-kernel table of a profiled
    solve ({kernel: (launches, total ms)}): the three passes each launch once
    per matvec.  Two byte counts: the floor the method must move (x and y,
    M, the stored spectrum octants once) and the three-pass traffic that adds
    the yz-transformed intermediate T (written, read and written, read)."""
    if not all(k in table and table[k][0] > 0 for k in MV_KERNELS):
        return None
    per = {k: table[k][1] / table[k][0] for k in MV_KERNELS}
    ms = sum(per.values())
    nx, ny, nz = p.nx, p.ny, p.nz
    N = nx * ny * nz
    L, Py, Pz = 2 * _smooth(nx), 2 * _smooth(ny), 2 * _smooth(nz)
    oct_ = 6 * (L // 2 + 1) * (Py // 2 + 1) * (Pz // 2 + 1)
    floor = 8 * (7 * N + oct_)
    three = sum(algorithmic(k, p, {})[1] for k in MV_KERNELS)
    gbs = lambda b: b / (ms * 1e-3) / 1e9
    return {"ms_per_matvec": ms, "kernels_ms": per, "floor_bytes": floor, "floor_gbs": gbs(floor),
            "three_pass_bytes": three, "three_pass_gbs": gbs(three), "frac_three_pass": gbs(three) / hbm_gbs,
            "peak_gbs": hbm_gbs}


def traffic(kernel: str, wname: str, plan_meta: dict):
    t = TRAFFIC.get(wname, {}).get(kernel)
    if t is None:
        return None
    kind, v = t
    if kind == "per_column":
        return v * (plan_meta["mean_j"] + 2)
    return v


def _smooth(n):
    def ok(v):
        for q in (2, 3, 5, 7):
            while v % q == 0:
                v //= q
        return v == 1
    while not ok(n):
        n += 1
    return n


# ---------------------------------------------------------------------------
# CPU oracle sample (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_iterations(wname: str, tol: float):
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(path):
        d = json.load(open(path)).get(wname, {}).get(f"{tol:g}")
        if d:
            return int(d["iters"]), "oracle GMRES count from tests/golden/oracle_iterations.json"
    return None, None


def oracle_solution(wname: str):
    """The oracle's stored solution of the workload (written by
    tests/golden/make_oracle_solutions.py, oracle GMRES to 1e-12), or None."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "oracle_solutions.json")
    if not os.path.exists(path):
        return None
    meta = json.load(open(path)).get(wname)
    if not meta or "sample" in meta:
        return None
    return np.load(os.path.join(ROOT, "tests", "golden", meta["file"]))


def solution_errors(w, ref) -> dict:
    """Relative 2-norm error and element-wise error (against the largest
    entry of the reference) of a solution."""
    import numpy as np
    return {"rel_err": float(np.linalg.norm(w - ref) / np.linalg.norm(ref)),
            "max_err": float(np.abs(w - ref).max() / np.abs(ref).max())}


class OracleSample:
    """Times the oracle's setup (generator spectra + full preconditioner
    build) once and its per-iteration work (FFT matvec, preconditioner apply,
    modified Gram-Schmidt against a 25-vector basis) on a few iterations."""

    def __init__(self, p):
        import numpy as np
        from oracle import operator as op
        from oracle import precond as pc
        self.np = np
        self.p = p
        t0 = time.perf_counter()
        self.k = op.background_k(p.k0, p.eps_bg)
        self.M = op.material(p.eps, p.eps_bg)
        self.b = op.rhs(p.eps, p.eps_bg, p.e_inc)
        self.spec = op.generator_spectra(p.nx, p.ny, p.nz, p.h, self.k)
        self.P = pc.Preconditioner(p.nx, p.ny, p.nz, p.h, self.k, self.M, p.boxes, p.homog, 1e-3)
        self.t_setup = time.perf_counter() - t0
        rng = np.random.default_rng(0)
        self.V = rng.standard_normal((25, self.b.size)) + 1j * rng.standard_normal((25, self.b.size))

    def iteration(self) -> float:
        from oracle import operator as op
        np = self.np
        t0 = time.perf_counter()
        z = self.P.apply(self.b)
        w = op.fft_matvec(z, self.M, self.spec).ravel()
        for i in range(self.V.shape[0]):
            h = np.vdot(self.V[i], w)
            w = w - h * self.V[i]
        return time.perf_counter() - t0

    def cycle(self, restart: int = 50) -> float:
        """Seconds of one full GMRES(restart) cycle of the oracle's own solver
        (oracle.gmres, right-preconditioned, from x = 0): restart iterations
        with the growing modified Gram-Schmidt, the cycle's update and its
        true-residual check."""
        from oracle import gmres as og
        from oracle import operator as op
        t0 = time.perf_counter()
        og.gmres(lambda v: op.fft_matvec(v, self.M, self.spec), self.b, self.P.apply, tol=1e-30,
                 restart=restart, max_iter=restart)
        return time.perf_counter() - t0

    def residual(self, w_gpu) -> float:
        from oracle import operator as op
        np = self.np
        r = self.b - op.fft_matvec(w_gpu, self.M, self.spec)
        return float(np.linalg.norm(r) / np.linalg.norm(self.b))


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# reference arm: the oracle alone
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, wname = workload(args.workload)
    iters, src = oracle_iterations(wname, args.tol)
    S = OracleSample(p)
    for _ in range(args.warmup):
        S.iteration()
    ts = [S.iteration() for _ in range(args.steps)]
    t_it = statistics.mean(ts)
    if iters is None:
        iters, src = 400, "assumed 400 iterations (no stored oracle count)"
    t_solve = S.t_setup + iters * t_it
    value = 1.0 / t_solve
    cores = cpu_cores()
    sample = (f"oracle setup (spectra + preconditioner build, {S.t_setup:.2f} s, once) + {args.steps} timed "
              f"iteration samples (FFT matvec + preconditioner apply + 25-vector MGS, mean {t_it:.3f} s); one solve "
              f"= setup + {iters} iterations ({src})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_it, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": wname, "precision": "fp64 (CPU oracle)", "tol": args.tol},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle_model", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1903_07884_gb300 import vie
    from paper_1903_07884_gb300.solver import Plan, to_device

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()

    p, wname = workload(args.workload)
    N = p.n_vox
    eps_d = to_device(p.eps, dev)
    e_d = to_device(p.e_inc, dev)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, tol=args.tol)

    def step():
        plan.set_permittivity(eps_d)
        plan.build()
        return plan.solve(e_d)

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = vie.vie_kernel_launches()
    times, infos = [], []
    w = None
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("bench_step")
        e0.record(plan.stream)
        w, info = step()
        e1.record(plan.stream)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
    torch.cuda.synchronize()
    barrier()
    launches = vie.vie_kernel_launches() - l0
    clk = clocks.stop()
    ms = aggregate_ms(statistics.mean(times), world, dist if world > 1 else None, dev)
    value = solves_per_s(ms, world)
    w_mixed = w.cpu().numpy()

    # plain FP64 GPU method on the same problem, same tolerance
    plan64 = Plan.for_problem(p, precision=vie.VIE_FP64, tol=args.tol)
    t64 = []
    w64 = None
    info64 = None
    for k in range(1 + args.fp64_steps):
        flush.fill_(k & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(plan64.stream)
        plan64.set_permittivity(eps_d)
        plan64.build()
        w64, info64 = plan64.solve(e_d)
        e1.record(plan64.stream)
        e1.synchronize()
        if k > 0:
            t64.append(e0.elapsed_time(e1))
    w64 = w64.cpu().numpy()
    plan64.close()
    diff = float(np.linalg.norm(w_mixed - w64) / np.linalg.norm(w64))

    # end to end through the host-buffer entry point (copies timed)
    eps_h = torch.from_numpy(np.ascontiguousarray(p.eps)).pin_memory()
    e_h = torch.from_numpy(np.ascontiguousarray(p.e_inc)).pin_memory()
    w_h = torch.empty(p.e_inc.shape, dtype=torch.complex128).pin_memory()
    te = []
    for k in range(1 + max(1, args.steps // 2)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(plan.stream)
        vie.vie_solve_host(plan.handle, eps_h.data_ptr(), e_h.data_ptr(), w_h.data_ptr())
        e1.record(plan.stream)
        e1.synchronize()
        if k > 0:
            te.append(e0.elapsed_time(e1))
    e2e_ms = aggregate_ms(statistics.mean(te), world, dist if world > 1 else None, dev)

    # per-kernel device time of one profiled solve (eager launches)
    vie.vie_profile_reset()
    vie.vie_profile_enable(True)
    step()
    torch.cuda.synchronize()
    vie.vie_profile_enable(False)
    table = vie.profile_table()
    vie.vie_profile_reset()
    total_prof = sum(t for _, t in table.values())
    top = sorted(table.items(), key=lambda kv: -kv[1][1])
    pk, pk_src = peaks()
    meta = plan_meta(p, infos[-1])
    roof = None
    for name, (cnt, tot) in top:
        a = algorithmic(name, p, meta)
        if a is None:
            continue
        kind, amount = a
        avg_ms = tot / cnt
        if kind == "hbm":
            ach = amount / (avg_ms * 1e-3) / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / pk["hbm_gbs"], "traffic": traffic(name, wname, meta), "share": tot / total_prof,
                    "avg_launch_ms": avg_ms, "launches": cnt, "peak_source": f"{pk_src} (MEASURED_PEAKS.json hbm_gbs)"}
        elif kind == "tensor":
            # tf32 peak = measured sustained bf16 x the nominal tf32 / bf16 ratio (1.1 / 2.25);
            # the 3xTF32 split issues three MMAs per algorithmic product
            tf32 = pk["bf16_tflops_sustained"] * 1.1 / 2.25
            ach = amount / (avg_ms * 1e-3) / 1e12
            roof = {"kernel": name, "bound": "tensor", "achieved": ach, "peak": tf32, "unit": "TFLOP/s",
                    "frac": ach / tf32, "traffic": None, "share": tot / total_prof,
                    "avg_launch_ms": avg_ms, "launches": cnt,
                    "peak_source": f"{pk_src} (bf16_tflops_sustained x 1.1/2.25 nominal tf32 ratio; 3xTF32 "
                                   "issues 3 MMAs per algorithmic product)"}
        else:
            ach = amount / (avg_ms * 1e-3) / 1e12
            f32 = name.endswith("_c64")
            alu = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
            roof = {"kernel": name, "bound": "alu", "achieved": ach, "peak": alu, "unit": "TFLOP/s",
                    "frac": ach / alu, "traffic": None, "share": tot / total_prof,
                    "avg_launch_ms": avg_ms, "launches": cnt,
                    "peak_source": ("FP32 FMA probe (8 independent FFMA chains" if f32 else
                                    "FP64 FMA probe (8 independent DFMA chains") + " x 8 warps x 152 SMs)"}
        break

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": wname, "grid": [p.nx, p.ny, p.nz], "h_um": p.h, "lambda_um": p.wavelength,
                       "precision": "mixed: c64 GMRES(50) in FP64 iterative refinement", "tol": args.tol,
                       "preconditioner": "1-level Chan-Olkin, real-mean homogenised, reduction tau=1e-3",
                       "l2": "512 MB buffer written between timed steps (outside the step events)",
                       "parallelism": f"replicas x{world}"},
            "iters": {"inner": infos[-1]["iters_inner"], "outer": infos[-1]["iters_outer"],
                      "reorth_passes": infos[-1]["reorth_passes"],
                      "fp64_fallback": infos[-1]["iters_fp64_fallback"]},
            "relres_fp64": infos[-1]["relres"], "kept_fraction": infos[-1]["kept_fraction"],
            "precond_bytes": infos[-1]["precond_bytes"],
            "fp64_gpu": {"value": 1000.0 / statistics.mean(t64) if t64 else None, "unit": UNIT,
                         "ms_per_solve": statistics.mean(t64) if t64 else None,
                         "iters": info64["iters_inner"], "relres_fp64": info64["relres"],
                         "rel_diff_mixed_vs_fp64": diff},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": solves_per_s(e2e_ms, world), "unit": UNIT,
                    "h2d_bytes_per_step": int(16 * N + 16 * 3 * N), "d2h_bytes_per_step": int(16 * 3 * N)},
            "roofline": roof,
            "autotune": vie.vie_plan_tuning(plan.handle),
            "matvec": matvec_summary(table, p, pk["hbm_gbs"]),
            "profile_ms": {k: round(v[1], 4) for k, v in top[:12]}}
    plan.close()

    if args.serving_n > 0:
        line["serving"] = run_serving(args.serving_n, args.inflight, args.budget_gb, args.tol, args.fp64_serial_s,
                                      args.fp64_serial_n, args.mixed_serial_n)

    ref = oracle_solution(wname)
    if ref is not None:
        line["accuracy"] = {"vs_oracle_solution": "tests/golden (oracle GMRES to relres 1e-12)",
                            "mixed": solution_errors(w_mixed, ref), "fp64_gpu": solution_errors(w64, ref)}
    else:
        smp = oracle_solution_sample(wname)
        if smp is not None:
            idx, wref = smp
            line["accuracy"] = {"vs_oracle_solution": f"tests/golden sample of {idx.size} entries (oracle GMRES "
                                                      "to relres 1e-12)",
                                "mixed": solution_errors(w_mixed.ravel()[idx], wref),
                                "fp64_gpu": solution_errors(w64.ravel()[idx], wref)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        S = OracleSample(p)
        restart = 50
        t_cyc = S.cycle(restart)
        iters, src = oracle_iterations(wname, args.tol)
        if iters is None:
            iters, src = infos[-1]["iters_inner"], "iteration count of the GPU FP64 solve"
        t_solve = S.t_setup + (iters / restart) * t_cyc
        line["cpu_baseline"] = {
            "value": 1.0 / t_solve, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": (f"the oracle's own solve of this workload, timed: setup {S.t_setup:.2f} s (generator spectra "
                       f"+ preconditioner build) and its first full GMRES({restart}) restart cycle {t_cyc:.2f} s "
                       f"({restart} iterations with the growing MGS, update and true residual); one solve = setup + "
                       f"{iters}/{restart} cycles ({iters} iterations: {src})")}
        acc = line.setdefault("accuracy", {})
        acc["oracle_relres_of_mixed_solution"] = S.residual(w_mixed)
        acc["oracle_relres_of_fp64_solution"] = S.residual(w64)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving(n_req: int, inflight: int, budget_gb: float, tol: float, fp64_limit_s: float, fp64_n: int = 16,
                mixed_serial_n: int = 0):
    """Replay the first n_req requests of the seeded serving stream (Poisson
    arrivals, 50/s) against the continuous-batching server; every request is
    submitted at its arrival time with host buffers and its latency runs from
    arrival to completion.  The same requests are then solved one by one with
    the plain FP64 GPU method (time-bounded by fp64_limit_s) and, if
    mixed_serial_n > 0, the first mixed_serial_n of them one by one with the
    same mixed method outside the server (what continuous batching gains)."""
    import numpy as np

    from paper_1903_07884_gb300 import inputs, vie
    from paper_1903_07884_gb300.solver import make_opts

    reqs = inputs.serving_stream(256)[:n_req]
    probs = [r.problem() for r in reqs]
    bufs = []
    for p in probs:
        bufs.append((np.ascontiguousarray(p.eps), np.ascontiguousarray(p.e_inc),
                     np.empty(p.e_inc.shape, dtype=np.complex128)))
    srv = vie.vie_server_create(int(budget_gb * (1 << 30)), inflight)
    t0 = time.perf_counter()
    tickets, t_arr, t_done, status = {}, {}, {}, {}
    infos = {}
    nxt = 0
    while len(t_done) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].t_arrival <= now:
            p = probs[nxt]
            eps, e, w = bufs[nxt]
            opts = make_opts(precision=vie.VIE_MIXED, tol=tol, boxes=p.boxes or None, homog=p.homog)
            st, t = vie.vie_server_submit(srv, p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, opts, eps.ctypes.data,
                                          e.ctypes.data, w.ctypes.data)
            tickets[t] = nxt
            t_arr[nxt] = reqs[nxt].t_arrival
            if st != vie.VIE_OK:
                t_done[nxt] = now
                status[nxt] = st
            nxt += 1
        for t, i in tickets.items():
            if i in t_done:
                continue
            st, info = vie.vie_server_poll(srv, t)
            if st != vie.VIE_PENDING:
                t_done[i] = time.perf_counter() - t0
                status[i] = st
                infos[i] = info
        time.sleep(0.0005)
    vie.vie_server_destroy(srv)
    lat = [1000.0 * (t_done[i] - t_arr[i]) for i in range(len(reqs))]
    span = max(t_done.values()) - min(t_arr.values())
    ok = sum(1 for s in status.values() if s in (vie.VIE_OK, vie.VIE_ENOCONV))
    converged = sum(1 for s in status.values() if s == vie.VIE_OK)
    unconverged = [{"request": i, "kind": reqs[i].kind, "grid": [reqs[i].nx, reqs[i].ny, reqs[i].nz],
                    "lambda_um": round(reqs[i].wavelength, 5), "relres": infos[i].relres,
                    "iters": infos[i].iters_inner, "status": int(status[i])}
                   for i in sorted(infos) if status.get(i) != vie.VIE_OK]
    out = {"requests": len(reqs), "stream_requests": 256,
           "cap": None if len(reqs) >= 256 else "first requests of the stream (default bench time); --serving-n 256 "
                                                "replays all of it",
           "ok": ok, "converged": converged, "unconverged": unconverged,
           "fp64_fallbacks": [{"request": i, "grid": [reqs[i].nx, reqs[i].ny, reqs[i].nz],
                               "lambda_um": round(reqs[i].wavelength, 5), "iters": infos[i].iters_inner,
                               "fp64_iters": infos[i].iters_fp64_fallback}
                              for i in sorted(infos) if infos[i].iters_fp64_fallback > 0],
           "solves_per_s": len(reqs) / span, "converged_solves_per_s": converged / span,
           "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "max_inflight": inflight, "budget_gb": budget_gb,
           "mean_iters": float(np.mean([infos[i].iters_inner for i in infos])) if infos else None,
           "max_relres": float(max(infos[i].relres for i in infos)) if infos else None}
    out["relres_all"] = "every served result's FP64 relative residual is <= max_relres"
    # plain FP64 GPU method, serially, on the first requests of the same stream
    # (at most fp64_n, time-bounded); each served result of those requests is
    # compared with its FP64 solution
    lat64, errs = [], []
    t_start = time.perf_counter()
    for i, p in enumerate(probs[:fp64_n]):
        if time.perf_counter() - t_start > fp64_limit_s:
            break
        eps, e, w_srv = bufs[i]
        w = np.empty(p.e_inc.shape, dtype=np.complex128)
        opts = make_opts(precision=vie.VIE_FP64, tol=tol, boxes=p.boxes or None, homog=p.homog)
        ts = time.perf_counter()
        plan = vie.vie_plan_create(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, opts, 0)
        vie.vie_solve_host(plan, eps.ctypes.data, e.ctypes.data, w.ctypes.data, allow_noconv=True)
        vie.vie_plan_destroy(plan)
        lat64.append(1000.0 * (time.perf_counter() - ts))
        if status.get(i) in (vie.VIE_OK, vie.VIE_ENOCONV):
            errs.append(float(np.linalg.norm(w_srv - w) / np.linalg.norm(w)))
    if mixed_serial_n > 0:
        latm, parts = [], []
        for i, p in enumerate(probs[:mixed_serial_n]):
            eps, e, _ = bufs[i]
            w = np.empty(p.e_inc.shape, dtype=np.complex128)
            opts = make_opts(precision=vie.VIE_MIXED, tol=tol, boxes=p.boxes or None, homog=p.homog)
            ts = time.perf_counter()
            plan = vie.vie_plan_create(p.nx, p.ny, p.nz, p.h, p.k0, p.eps_bg, opts, 0)
            tc = time.perf_counter()
            info = vie.vie_solve_host(plan, eps.ctypes.data, e.ctypes.data, w.ctypes.data, allow_noconv=True)
            vie.vie_plan_destroy(plan)
            latm.append(time.perf_counter() - ts)
            parts.append((tc - ts, info.t_setup_ms / 1e3, info.t_solve_ms / 1e3))
        out["mixed_serial"] = {"requests": len(latm), "solves_per_s": len(latm) / sum(latm),
                               "seconds": {"plan_create": sum(a for a, _, _ in parts),
                                           "precond_build": sum(b for _, b, _ in parts),
                                           "solve_incl_build": sum(c for _, _, c in parts), "total": sum(latm)},
                               "note": "the same mixed method, each request alone through vie_plan_create + "
                                       "vie_solve_host, first requests of the same stream"}
    if lat64:
        out["fp64_serial"] = {"requests": len(lat64), "solves_per_s": len(lat64) / (sum(lat64) / 1000.0),
                              "p50_ms": float(np.percentile(lat64, 50)), "p99_ms": float(np.percentile(lat64, 99)),
                              "time_bound_s": fp64_limit_s,
                              "note": "each request alone, no queueing; first requests of the same stream"}
        out["max_rel_err_vs_fp64"] = max(errs) if errs else None
        out["rel_err_vs_fp64_requests"] = len(errs)
    return out


def run_batch(args):
    """Directional-coupler batch (2048x48x8 grid, h = 0.025 um, two 16x8 Si
    cores in SiO2 with one preconditioner box each): --batch-n wavelengths
    spaced evenly over 1.50-1.60 um solved together through vie_solve_batch
    (one lockstep set: per step one captured graph, the Arnoldi kernels as
    single launches over the work-list of all plans), against the same
    solves one after another.  One step = permittivity + preconditioner
    build of every plan + the batch solve.  Prints one bench line."""
    import numpy as np
    import torch

    from paper_1903_07884_gb300 import inputs, vie
    from paper_1903_07884_gb300.solver import Plan, to_device

    torch.cuda.set_device(0)
    lams = inputs.coupler_wavelengths(args.batch_n)
    probs = [inputs.workload_coupler(wavelength=float(l)) for l in lams]
    p0 = probs[0]
    plans = [Plan.for_problem(p, precision=vie.VIE_MIXED, tol=args.tol) for p in probs]
    eps = [to_device(p.eps) for p in probs]
    es = [to_device(p.e_inc) for p in probs]
    ws = [torch.empty_like(e) for e in es]

    def prepare():
        for pl, e in zip(plans, eps):
            pl.set_permittivity(e)
            pl.build()

    def batch_step():
        prepare()
        return vie.vie_solve_batch([pl.handle for pl in plans], [e.data_ptr() for e in es],
                                   [w.data_ptr() for w in ws])

    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        batch_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = vie.vie_kernel_launches()
    times, infos = [], None
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = batch_step()      # synchronous: every plan's build and the batch solve are done on return
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = vie.vie_kernel_launches() - l0
    clk = clocks.stop()
    ms = statistics.mean(times)
    value = len(plans) * 1000.0 / ms
    w_batch = [w.cpu().numpy() for w in ws]
    # the same solves one after another
    ts = []
    seq_equal = True
    for k in range(2):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        outs = []
        for pl, e in zip(plans, eps):
            pl.set_permittivity(e)
            pl.build()
        for pl, e in zip(plans, es):
            w, _ = pl.solve(e)
            outs.append(w)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
        seq_equal = seq_equal and all(np.array_equal(o.cpu().numpy(), wb) for o, wb in zip(outs, w_batch))
    ms_seq = statistics.mean(ts)
    # per-kernel device time of one profiled batch step (eager launches)
    vie.vie_profile_reset()
    vie.vie_profile_enable(True)
    batch_step()
    torch.cuda.synchronize()
    vie.vie_profile_enable(False)
    table = vie.profile_table()
    vie.vie_profile_reset()
    total_prof = sum(t for _, t in table.values())
    top = sorted(table.items(), key=lambda kv: -kv[1][1])
    pk, pk_src = peaks()
    meta = plan_meta(p0, infos[0].as_dict())
    meta["plans_per_launch"] = len(plans)
    roof = None
    for name, (cnt, tot) in top:
        a = algorithmic(name, p0, meta)
        if a is None or a[0] != "hbm":
            continue
        avg_ms = tot / cnt
        ach = a[1] / (avg_ms * 1e-3) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": None, "share": tot / total_prof, "avg_launch_ms": avg_ms,
                "launches": cnt, "peak_source": f"{pk_src} (MEASURED_PEAKS.json hbm_gbs)"}
        break
    # accuracy: each solution's FP64 residual recomputed by the CPU oracle on a
    # sample of wavelengths, and the first one against the stored oracle sample
    acc = {"relres_fp64_max": max(i.relres for i in infos)}
    if not args.no_cpu_baseline:
        chk = sorted({0, len(plans) // 2, len(plans) - 1})
        rr = {}
        for i in chk:
            S = OracleResidual(probs[i])
            rr[f"{lams[i]:.4f}"] = S.residual(w_batch[i])
        acc["oracle_relres_sampled"] = rr
        ref = oracle_solution_sample(f"coupler_2048x48x8_2boxes_lambda{lams[0]:.2f}")
        if ref is not None:
            idx, wref = ref
            wv = w_batch[0].ravel()[idx]
            acc["lambda0_vs_oracle_sample"] = {"rel_err": float(np.linalg.norm(wv - wref) / np.linalg.norm(wref)),
                                               "max_err": float(np.abs(wv - wref).max() / np.abs(wref).max()),
                                               "entries": int(idx.size)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": f"coupler_batch_{len(plans)}x2048x48x8_2boxes", "grid": [p0.nx, p0.ny, p0.nz],
                       "wavelengths_um": [round(float(l), 5) for l in lams], "tol": args.tol,
                       "precision": "mixed: c64 GMRES in FP64 iterative refinement",
                       "preconditioner": "block-diagonal 1-level Chan-Olkin, one box per core, tau=1e-3",
                       "l2": "512 MB buffer written between timed steps (outside the step events)"},
            "iters": [i.iters_inner for i in infos], "clocks": clk, "gpu_launches": int(launches),
            "sequential": {"ms_per_step": ms_seq, "value": len(plans) * 1000.0 / ms_seq,
                           "bitwise_equal_to_batch": bool(seq_equal)},
            "accuracy": acc, "roofline": roof, "autotune": vie.vie_plan_tuning(plans[0].handle),
            "profile_ms": {k: round(v[1], 4) for k, v in top[:12]}}
    for pl in plans:
        pl.close()
    print(json.dumps(line))
    return 0


class OracleResidual:
    """The CPU oracle's FP64 relative residual of a solution (FFT matvec)."""

    def __init__(self, p):
        from oracle import operator as op
        self.k = op.background_k(p.k0, p.eps_bg)
        self.M = op.material(p.eps, p.eps_bg)
        self.b = op.rhs(p.eps, p.eps_bg, p.e_inc)
        self.spec = op.generator_spectra(p.nx, p.ny, p.nz, p.h, self.k)

    def residual(self, w) -> float:
        import numpy as np
        from oracle import operator as op
        r = self.b - op.fft_matvec(w, self.M, self.spec)
        return float(np.linalg.norm(r) / np.linalg.norm(self.b))


def oracle_solution_sample(wname: str):
    """(indices, values) of a stored sampled oracle solution, or None."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "oracle_solutions.json")
    if not os.path.exists(path):
        return None
    meta = json.load(open(path)).get(wname)
    if not meta or "sample" not in meta:
        return None
    d = np.load(os.path.join(ROOT, "tests", "golden", meta["file"]))
    return d["idx"], d["w"]


def plan_meta(p, info):
    """Block sizes of the preconditioner for the work formulas: every box of
    the workloads has the same cross-section, so the stored block and
    discarded-slot counts divide evenly over the boxes."""
    boxes = p.boxes or [(0, 0, 0, p.nx, p.ny, p.nz)]
    m = 3 * boxes[0][4] * boxes[0][5]
    nblk = info["precond_blocks"] / len(boxes)
    ndisc = info["precond_discarded"] / len(boxes)
    # mean step index j over the Arnoldi launches: every refinement step is
    # one cycle of k columns, which takes the steps j = 0..k
    its, outer = info["iters_inner"], max(1, info["iters_outer"])
    per = its / outer
    mean_j = per / 2.0
    # the representative takes a slot of its own unless it is kept
    return {"m": m, "nblk": nblk, "nhalf": max(1.0, nblk - 1), "ndisc": ndisc, "nboxes": len(boxes),
            "mean_j": mean_j}


def run_study(args):
    """Qualitative studies of the method on the GPU path (FP64 GMRES(50) at
    tolerance 1e-4, as in the paper's iteration plots; no memory reduction):

    bragg  - Sec. 5.2: iterations of the three homogenisation variants
             (mode, mean, real part of the mean) against the grating length
             (number of periods, width step 50 nm) and against the fill D/N as
             the corrugation depth grows (100 periods);
    bragg_bench_shape - the same two sweeps on the benchmark grating's shape
             (24x8 voxels, core 16/12, period 32, two x-boxes; 64 periods for
             the depth sweep);
    length - Sec. 3 and 4: iterations of unpreconditioned GMRES against the
             length of a Si wire in air, beside the 1-level preconditioner;
    disk   - Sec. 5.3.1: disk resonators of radius 1-5 um beside a bus, with
             the blocked-circulant preconditioner (reduced 1-level bus box,
             2-level disk box, modal M~) and without one (capped at 6000).
    Prints one JSON line with the rows."""
    import numpy as np

    from paper_1903_07884_gb300 import inputs, vie
    from paper_1903_07884_gb300.solver import Plan, to_device

    def iters(p, homog=3, precond=vie.VIE_PREC_CIRCULANT, reduce_tol=0.0, max_iter=20000, full=False):
        plan = Plan.for_problem(p, precision=vie.VIE_FP64, tol=1e-4, reduce_tol=reduce_tol, homog=homog,
                                precond=precond, max_iter=max_iter, restart=args.study_restart)
        plan.set_permittivity(to_device(p.eps))
        t0 = time.perf_counter()
        _, info = plan.solve(to_device(p.e_inc), allow_noconv=True)
        secs.append(time.perf_counter() - t0)
        plan.close()
        if full:
            return info
        return info["iters_inner"], info["relres"]

    secs = []

    rows = []
    names = {1: "mode", 2: "mean", 3: "real_mean"}
    if args.study == "bragg":
        # grating box 20 voxels (500 nm) wide, 8 (200 nm) high, period 14 voxels
        # (350 nm), h = 25 nm, lambda = 1.55 um, Si in SiO2, one box
        wide, period = 20, 14
        for nper in (10, 20, 40, 80, 160, 320):
            p = inputs.bragg_grating(nper * period, wide, 8, 0.025, 1.55, wide=wide, narrow=wide - 2, period=period,
                                     nboxes=1, name=f"bragg_nper{nper}")
            for v in (1, 2, 3):
                it, rr = iters(p, homog=v)
                rows.append({"sweep": "length", "n_per": nper, "dW_nm": 50, "variant": names[v], "iters": it,
                             "relres": rr})
        for dw in (0, 2, 4, 6, 8, 10, 12):
            p = inputs.bragg_grating(100 * period, wide, 8, 0.025, 1.55, wide=wide, narrow=wide - dw, period=period,
                                     nboxes=1, name=f"bragg_dw{dw}")
            x = np.arange(p.nx)
            fill = float(np.mean(np.where((x % period) < period // 2, wide, wide - dw)) / wide)
            for v in (1, 2, 3):
                it, rr = iters(p, homog=v)
                rows.append({"sweep": "depth", "n_per": 100, "dW_nm": 25 * dw, "D_over_N": fill,
                             "variant": names[v], "iters": it, "relres": rr})
    elif args.study == "bragg_bench_shape":
        # the benchmark grating's shape: 24x8 cross-section, core 16 voxels
        # (400 nm) wide with 12-voxel narrow sections, period 32 (800 nm),
        # h = 25 nm, lambda = 1.55 um, Si in SiO2, two x-boxes
        wide, period = 16, 32
        for nper in (8, 16, 32, 64, 128):
            p = inputs.bragg_grating(nper * period, 24, 8, 0.025, 1.55, wide=wide, narrow=wide - 4, period=period,
                                     name=f"bragg24_nper{nper}")
            for v in (1, 2, 3):
                it, rr = iters(p, homog=v)
                rows.append({"sweep": "length", "n_per": nper, "dW_nm": 100, "variant": names[v], "iters": it,
                             "relres": rr})
        for dw in (0, 2, 4, 6, 8, 10):
            p = inputs.bragg_grating(64 * period, 24, 8, 0.025, 1.55, wide=wide, narrow=wide - dw, period=period,
                                     name=f"bragg24_dw{dw}")
            x = np.arange(p.nx)
            fill = float(np.mean(np.where((x % period) < period // 2, wide, wide - dw)) / wide)
            for v in (1, 2, 3):
                it, rr = iters(p, homog=v)
                rows.append({"sweep": "depth", "n_per": 64, "dW_nm": 25 * dw, "D_over_N": fill,
                             "variant": names[v], "iters": it, "relres": rr})
    elif args.study == "disk":
        # Sec. 5.3.1, Table disk: 20 nm voxels, 220 nm slab, 400 nm bus, 200 nm
        # gap; reduced 1-level bus box + 2-level disk box with the modal M~
        for r_um in [float(v) for v in args.study_radii.split(",")]:
            p = inputs.disk_resonator(int(round(r_um / 0.02)), name=f"disk_r{r_um}")
            row = {"radius_um": r_um, "grid": [p.nx, p.ny, p.nz], "homog": args.study_homog}
            info = iters(p, homog=args.study_homog, reduce_tol=1e-3, max_iter=args.study_max_iter, full=True)
            row.update(prec_iters=info["iters_inner"], prec_relres=info["relres"],
                       build_s=round(info["t_setup_ms"] / 1e3, 3), prec_solve_s=round(secs[-1], 3),
                       precond_mb=round(info["precond_bytes"] / 2 ** 20, 1))
            if not args.study_no_baseline:
                it0, r0 = iters(p, precond=vie.VIE_PREC_NONE, max_iter=6000)
                row.update(noprec_iters=it0, noprec_relres=r0, noprec_solve_s=round(secs[-1], 3))
            rows.append(row)
    else:
        for nx in (128, 256, 512, 1024, 2048):
            p = inputs.straight_guide(nx, 16, 8, 0.025, 1.55, name=f"wire_{nx}")
            it0, r0 = iters(p, precond=vie.VIE_PREC_NONE)
            it1, r1 = iters(p)
            rows.append({"nx": nx, "length_um": nx * 0.025, "unpreconditioned_iters": it0, "relres0": r0,
                         "preconditioned_iters": it1, "relres1": r1})
    print(json.dumps({"study": args.study, "tol": 1e-4, "precision": "fp64", "restart": args.study_restart,
                      "solve_seconds": [round(s, 3) for s in secs], "rows": rows}))
    return 0


def run_profile_case(args):
    """Create a plan and solve the workload once in mixed precision: the
    plan creation (outside the bench's timed step) and then the launch
    sequence of one bench step, without the timing, comparison and serving
    legs, so that an ncu capture of it stays short."""
    from paper_1903_07884_gb300 import vie
    from paper_1903_07884_gb300.solver import Plan, to_device
    p, wname = workload(args.workload)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, tol=args.tol)
    plan.set_permittivity(to_device(p.eps))
    _, info = plan.solve(to_device(p.e_inc))
    plan.close()
    print(json.dumps({"profile_case": wname, "iters": info["iters_inner"], "relres": info["relres"],
                      "launches": vie.vie_kernel_launches()}))
    return 0


def run_profile_request(args):
    """Create the plan of request args.profile_request of the 256-request
    serving stream and run one mixed solve of it, nothing else (for ncu
    captures of the kernels a serving request takes).  Prints one JSON line
    (not a bench line)."""
    from paper_1903_07884_gb300 import inputs, vie
    from paper_1903_07884_gb300.solver import Plan, to_device
    r = inputs.serving_stream(256)[args.profile_request]
    p = r.problem()
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, tol=args.tol)
    plan.set_permittivity(to_device(p.eps))
    _, info = plan.solve(to_device(p.e_inc))
    plan.close()
    print(json.dumps({"profile_request": args.profile_request, "grid": [p.nx, p.ny, p.nz], "kind": r.kind,
                      "iters": info["iters_inner"], "relres": info["relres"]}))
    return 0


def run_precond2_case(args):
    """Blocked disk preconditioner (reduced 1-level bus box + 2-level disk box,
    3 um radius, 20 nm voxels, complex-FP32 apply): per-kernel device times of
    10 applies after 3 warm-up applies, and the bandwidth the 2-level block
    product reaches (its stored inverses, 22 801 blocks of 33 x 33, exceed L2).
    Prints one JSON line (not a bench line)."""
    import torch

    from paper_1903_07884_gb300 import inputs, vie
    from paper_1903_07884_gb300.solver import Plan, to_device
    p = inputs.disk_resonator(150)
    plan = Plan.for_problem(p, precision=vie.VIE_MIXED, reduce_tol=1e-3, homog=1)
    plan.set_permittivity(to_device(p.eps))
    plan.build()
    r = to_device(inputs.random_field((3, p.nz, p.ny, p.nx), seed=5))
    for _ in range(3):
        plan.precond(r, vie.VIE_MIXED)
    torch.cuda.synchronize()
    reps = 10
    vie.vie_profile_reset()
    vie.vie_profile_enable(True)
    for _ in range(reps):
        plan.precond(r, vie.VIE_MIXED)
    torch.cuda.synchronize()
    vie.vie_profile_enable(False)
    table = vie.profile_table()
    vie.vie_profile_reset()
    plan.close()
    _, _, _, n, ny, nz, _ = p.boxes[1]
    m2 = 3 * nz
    slots = (n // 2 + 1) * (ny // 2 + 1)
    algo = 8 * (slots * m2 * m2 + 2 * m2 * n * ny)     # inverses once, spectra in and out once
    launches, tot = table["block_gemv2_c64"]
    per_ms = tot / launches
    pk, pk_src = peaks()
    ach = algo / (per_ms * 1e-3) / 1e9
    print(json.dumps({"precond2_case": f"disk r=3um {p.nx}x{p.ny}x{p.nz}, disk box {n}x{ny}x{nz}",
                      "block_gemv2_c64": {"launches": launches, "avg_ms": round(per_ms, 5),
                                          "algorithmic_bytes": algo, "achieved_gbs": round(ach, 1),
                                          "peak_gbs": pk["hbm_gbs"], "peak_source": pk_src,
                                          "frac": round(ach / pk["hbm_gbs"], 3)},
                      "apply_kernels_ms_per_apply": {k: round(v[1] / reps, 4) for k, v in
                                                     sorted(table.items(), key=lambda kv: -kv[1][1])}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gvie", choices=["gvie", "reference"])
    ap.add_argument("--workload", default="long_straight",
                    help="long_straight (default), small_straight, bragg, coupler, or coupler_batch")
    ap.add_argument("--batch-n", type=int, default=16, help="coupler_batch: number of wavelengths")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-n", type=int, default=32,
                    help="requests of the 256-request serving stream to replay (0 = skip; the default keeps the "
                         "bench within minutes, 256 replays the whole stream)")
    ap.add_argument("--inflight", type=int, default=32)
    ap.add_argument("--budget-gb", type=float, default=220.0)
    ap.add_argument("--fp64-serial-s", type=float, default=30.0, help="time bound of the serial FP64 serving leg")
    ap.add_argument("--fp64-serial-n", type=int, default=16, help="requests of the serial FP64 serving leg")
    ap.add_argument("--mixed-serial-n", type=int, default=0,
                    help="requests solved one by one with the mixed method outside the server (0 = skip)")
    ap.add_argument("--profile-request", type=int, default=None,
                    help="one mixed solve of that request of the serving stream and nothing else (for ncu captures)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one mixed solve of the workload and nothing else (for ncu captures; prints no bench line)")
    ap.add_argument("--study", choices=["bragg", "bragg_bench_shape", "length", "disk"], default=None,
                    help="qualitative iteration studies (prints one JSON line; not a bench line)")
    ap.add_argument("--precond2-case", action="store_true",
                    help="time the blocked 2-level preconditioner apply of a 3 um disk (prints no bench line)")
    ap.add_argument("--study-restart", type=int, default=50, help="GMRES restart length of the studies")
    ap.add_argument("--study-radii", default="1,2,3,4,5", help="disk study: radii in um")
    ap.add_argument("--study-homog", type=int, default=1, help="disk study: homogenisation variant (1 mode)")
    ap.add_argument("--study-no-baseline", action="store_true", help="disk study: skip the unpreconditioned solves")
    ap.add_argument("--study-max-iter", type=int, default=20000, help="disk study: cap of the preconditioned solves")
    args = ap.parse_args()
    if args.study:
        return run_study(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.precond2_case:
        return run_precond2_case(args)
    if args.profile_request is not None:
        return run_profile_request(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "coupler_batch":
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
