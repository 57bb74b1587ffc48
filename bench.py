#!/usr/bin/env python
"""Throughput of the HIF-IE hot path on GB300.

One step = factor A (Algorithm 4.1, second-kind modifications of Sec. 4.4) in
FP32 and solve all right-hand sides to relative residual 1e-10 by iterative
refinement preconditioned with the factorization, residuals from the exact
direct-sum operator (tensor cores on exact 8-bit digits of the FP64 table and
sources, FP64-class accuracy).  Workload: 2D second-kind volume IE on the unit square,
n = 1024 (N = 1,048,576), kernel -log(r)/(2 pi), a = 1, b = c = 1 + 0.5 phi
(16 random-phase cosines), eps = 1e-6, 8 Gaussian right-hand sides.

value = (all ranks) N * nrhs / (time per step): unknowns solved to 1e-10 per
second, factorization included.  Multi-GPU runs are independent replicas
(weak scaling; the single-problem path has no data-parallel split).

``--impl reference`` times the CPU oracle (plain numpy, FP64) on a bounded
sample of the same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "factor s + solve DOF/s on GB300 at stated rel. err; FP32+refine/batched vs FP64"
UNIT = "DOF/s"
TOL = 1e-10
ORACLE_SAMPLE_N = 64
ORACLE_SCALING_N = (32, 64)


def workload_config(n, nrhs, eps):
    return {
        "workload": (f"2D second-kind volume IE, unit square, n={n} (N={n * n}), kernel -log(r)/2pi, "
                     f"a=1, b=c=1+0.5*phi (16 random-phase cosines, seed 1002), eps={eps:g}, "
                     f"{nrhs} Gaussian RHS (seed 1003); FP32 HIF-IE factorization + iterative refinement "
                     f"to rel. residual {TOL:g} against the exact direct sum (tensor cores, exact 8-bit digits, "
                     f"FP64-class accuracy)"),
        "n": n, "N": n * n, "nrhs": nrhs, "eps": eps, "tol": TOL,
        "l2": "inputs larger than L2 (factor data and the 8-RHS vectors exceed the 129 MB L2)",
    }


# ----------------------------------------------------------------- oracle --

def oracle_sample(n=ORACLE_SAMPLE_N, eps=1e-6):
    """The oracle as it stands on a bounded sample: FP64 sequential HIF-IE
    factorization + iterative refinement to 1e-10 with the oracle's direct-sum
    matvec, one right-hand side."""
    import numpy as np
    import hif_inputs as hi
    from oracle import hifie, kernels, krylov
    pb = hi.volume_problem(n, 2, smooth_seed=1002, rhs_seed=1003, nrhs=1)
    t0 = time.perf_counter()
    F = hifie.factor(pb.points, pb.weights, pb.a, pb.b, pb.c, 0, eps, pb.proxy)
    op = kernels.Operator(pb.points, pb.weights, pb.a, pb.b, pb.c, 0)
    u, its, hist = krylov.refine(op.matvec, pb.f[:, 0], F.solve, tol=TOL)
    dt = time.perf_counter() - t0
    return {"seconds": dt, "N": pb.N, "nrhs": 1, "value": pb.N / dt, "iters": its, "relres": float(hist[-1]),
            "sample": (f"oracle FP64 HIF-IE factor + iterative refinement to {TOL:g} (oracle direct-sum residual), "
                       f"1 RHS, n={n} grid (N={pb.N}) of the same IE; value = N/time")}


def run_oracle_subprocess(n=ORACLE_SAMPLE_N):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample-json", str(n)],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- GPU arm ---

def alu_peaks(peaks):
    """FP32 and FP64 SIMT peaks from the unit counts and the measured maximum
    SM clock: 152 SMs x 128 FP32 lanes (one FMA = 2 flop per clock) and
    152 SMs x 2 FP64 FMA per clock."""
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return {"fp32": 152 * 128 * 2 * mhz * 1e6 / 1e12, "fp64": 152 * 2 * 2 * mhz * 1e6 / 1e12}


def kernel_rooflines(prof, peaks, precision):
    """One entry per kernel family of a profiled step: achieved work / event
    time against the peak of the unit that bounds it (Sec. 8 rooflines:
    fold / ID / elimination on the FP32 or FP64 SIMT pipes, pivot steps and
    sweeps on HBM, the direct sum on the tensor pipe)."""
    alu = alu_peaks(peaks)
    hbm = peaks.get("hbm_gbs", 6800.0)
    tens = peaks.get("bf16_tflops_sustained", 1700.0)
    simt = alu["fp32"] if precision == "fp32" else alu["fp64"]
    simt_name = f"{precision} SIMT pipe, derived from unit counts x sm_max_mhz"
    bound = {"fold_kernel": ("alu", simt, simt_name), "id_kernel": ("alu", simt, simt_name),
             "elim_kernel": ("alu", simt, simt_name), "big_elim_batch": ("alu", simt, simt_name),
             "big_qr_step": ("hbm", hbm, "MEASURED_PEAKS.json hbm_gbs"),
             "big_ygen_kernel": ("hbm", hbm, "MEASURED_PEAKS.json hbm_gbs"),
             "sweep": ("hbm", hbm, "MEASURED_PEAKS.json hbm_gbs"),
             "direct_sum": ("tensor", tens, "MEASURED_PEAKS.json bf16_tflops_sustained"),
             "direct_sum_short": ("tensor", tens, "MEASURED_PEAKS.json bf16_tflops_sustained")}
    out = []
    for name, e in prof.items():
        if not e["ranges"]:
            continue
        t = e["ms"] / 1000.0
        row = {"kernel": name, "ranges": e["ranges"], "seconds": t}
        if name in bound and t > 0:
            kind, peak, src = bound[name]
            if kind == "hbm":
                ach = e["bytes"] / t / 1e9
                row.update(bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak,
                           algorithmic_bytes=e["bytes"], peak_source=src)
            else:
                ach = e["flops"] / t / 1e12
                row.update(bound=kind, achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                           algorithmic_flops=e["flops"], peak_source=src)
        out.append(row)
    return out


def max_over_ranks(t_local, world, device):
    """The slowest rank's time: every rank's timed region ends at a barrier
    and the job's throughput is counted against the maximum."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, t_max):
    """Whole-job throughput of independent replicas (weak scaling): every
    rank processes the same units; no collective in the data path."""
    return world * units_per_rank / t_max


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    from paper_1307_2666_gb300 import hif as H

    dev = torch.device(f"cuda:{local}")
    n, nrhs, eps = args.n, args.nrhs, args.eps
    pb = hi.volume_problem(n, 2, smooth_seed=1002, rhs_seed=1003, nrhs=nrhs)
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev)
    pts, w, a, b, c = T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)
    F = T(pb.f.T).t()                                    # column-major N x nrhs on the device
    N = pb.N
    stats = {}

    def step(precision="fp32"):
        fac = P.Factorization(pts, w, a, b, c, 0, eps, precision=precision)
        u, its, rel = fac.solve_refined(F, tol=TOL, method="ir")
        stats.update(iters=its, relres=rel, top=fac.stats()["top_size"], mf=fac.stats()["factor_bytes"],
                     t_factor=fac.stats()["factor_seconds"])
        fac.close()
        return u

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = H.hif_kernel_launches()
    H.hif_kernel_timing(True)                            # CUDA events around the dominant kernel
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record()
    for _ in range(args.steps):
        step()
    ev1.record()
    barrier()
    launches = H.hif_kernel_launches() - launches0
    tc_ms, tc_launches = H.hif_kernel_timing(False)
    clocks = sampler.stop()
    t_max = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0, world, dev)
    ms_per_step = 1000.0 * t_max / args.steps
    value = job_value(N * nrhs * args.steps, world, t_max)

    # ---- solve-only split of one step, for the report
    fac = P.Factorization(pts, w, a, b, c, 0, eps, precision="fp32")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    u, its, rel = fac.solve_refined(F, tol=TOL, method="ir")
    e1.record()
    torch.cuda.synchronize()
    t_solve = e0.elapsed_time(e1) / 1000.0
    t_factor = fac.stats()["factor_seconds"]
    st32 = fac.stats()
    fp32_stats = dict(top=st32["top_size"], mf=st32["factor_bytes"], sym=st32["symmetric_problems"] > 0,
                      rows=st32["proxy_rows"])

    # ---- dominant kernel: the tensor-core direct sum (one launch per 8 RHS),
    # timed with CUDA events on its own stream inside the timed steps above
    y = torch.empty_like(F)
    reps = 2
    e0.record()
    for _ in range(reps):
        P.hif_matvec(fac.h, 0, F, y)
    e1.record()
    torch.cuda.synchronize()
    t_mv = e0.elapsed_time(e1) / 1000.0 / reps
    fac.close()
    peaks = measured_peaks()
    groups = -(-nrhs // 8)
    # algorithmic work of the method (Sec. 8 roofline of the direct sum):
    # 2 N^2 flops per right-hand side; the kernel forms them from exact 8-bit
    # digit products, 256 BF16 MACs per (target, source) pair and 8 RHS
    flops_launch = 2.0 * N * N * min(nrhs, 8)
    digit_flops_launch = 512.0 * N * N * min(nrhs, 8) / 8.0
    t_launch = (tc_ms / 1000.0 / tc_launches) if tc_launches else float("nan")
    achieved = flops_launch / t_launch / 1e12
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    fp64_pipe = alu_peaks(peaks)["fp64"]
    roofline = {"kernel": "tc_conv_kernel (direct sum on tcgen05 tensor cores, exact 8-bit digits)",
                "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside the step)"
                                if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s sustained"),
                "algorithmic_per_launch": f"2 N^2 flops per RHS x {min(nrhs, 8)} RHS = {flops_launch:.3e} flop",
                "launch_seconds": t_launch, "launches_timed": tc_launches, "traffic": None,
                "digit_mac_tflops": digit_flops_launch / t_launch / 1e12,
                "digit_mac_occupancy": digit_flops_launch / t_launch / 1e12 / peak,
                "fp64_pipe_peak_tflops": fp64_pipe, "vs_fp64_pipe": achieved / fp64_pipe,
                "matvec_seconds": t_mv, "matvec_launches_per_call": groups}

    # ---- every hot kernel family of one more step, timed per launch with
    # CUDA events (outside the timed region)
    H.hif_kernel_profile(True)
    step()
    torch.cuda.synchronize()
    prof = H.hif_kernel_profile(False)
    roofline_kernels = kernel_rooflines(prof, peaks, "fp32")

    # ---- FP64 factorization path for comparison (one step)
    fp64 = None
    if args.compare_fp64:
        e0.record()
        step("fp64")
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1000.0
        fp64 = {"ms_per_step": 1000 * t64, "value": N * nrhs / t64, "iters": stats.get("iters"),
                "relres": stats.get("relres"), "top_size": stats.get("top"), "t_factor_s": stats.get("t_factor")}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    hp = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64).pin_memory()
    h_pts, h_w, h_a, h_b, h_c = hp(pb.points), hp(pb.weights), hp(pb.a), hp(pb.b), hp(pb.c)
    h_f = hp(pb.f.T).t()
    h_u = torch.empty((nrhs, N), dtype=torch.float64).pin_memory().t()
    opt = H.hif_options_default(2)
    opt.precision = 1
    barrier()
    t0 = time.perf_counter()
    e0.record()
    hdl = H.hif_factor(h_pts, h_w, h_a, h_b, h_c, 0, eps, opt)
    H.hif_solve_refined(hdl, 0, h_f, h_u, TOL, 50, 0)
    e1.record()
    torch.cuda.synchronize()
    t_e2e = max(e0.elapsed_time(e1) / 1000.0, time.perf_counter() - t0)
    H.hif_destroy(hdl)
    h2d = (pb.points.nbytes + 4 * pb.weights.nbytes + pb.f.nbytes)
    d2h = pb.f.nbytes
    e2e = {"value": N * nrhs / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "seconds": t_e2e}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        runs = [run_oracle_subprocess(nn) for nn in ORACLE_SCALING_N]
        s = runs[-1]
        cpu = {"value": s["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": s["sample"],
               "seconds": s["seconds"], "iters": s["iters"], "relres": s["relres"],
               "same_config": False,
               "config_note": (f"the oracle runs n={ORACLE_SCALING_N[-1]} (N={s['N']}), 1 RHS; the GPU line runs "
                               f"n={n} (N={N}), {nrhs} RHS. The oracle's dense Schur store makes it O(N^2) in "
                               f"memory and worse in time, so DOF/s falls with N; the scaling entries show it."),
               "scaling": [{"n": nn, "N": r["N"], "seconds": r["seconds"], "value": r["value"]}
                           for nn, r in zip(ORACLE_SCALING_N, runs)]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 factor; residual bf16 digits, exact int sums", "data": "synthetic",
            "config": dict(workload_config(n, nrhs, eps), parallelism=f"replicas x{world}"),
            "t_factor_s": t_factor, "t_solve_s": t_solve, "refine_iters": its, "relres": rel,
            "top_size": fp32_stats["top"], "factor_bytes": fp32_stats["mf"],
            "symmetric_compression": fp32_stats["sym"], "proxy_rows": fp32_stats["rows"],
            "fp64_path": fp64, "roofline": roofline, "roofline_kernels": roofline_kernels,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batched(args):
    """Independent problems in one handle: P 2D second-kind IEs with n drawn
    from {32, 48, ..., 256} (seed 1004), b = c = 1 + 0.5 phi_p (seed 2000 + p),
    eps 1e-6, 4 Gaussian RHS each (seed 3000 + p); one step
    = factor all problems in one batched handle + refine all RHS to 1e-10.
    Reported next to the same problems factored and refined one handle at a
    time (FP64, the plain path) and to the batched handle in FP32."""
    import numpy as np
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    from paper_1307_2666_gb300 import hif as H
    dev = torch.device(f"cuda:{local}")
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev)
    sizes = hi.batched_sizes(args.problems, seed=1004)
    pbs = [hi.volume_problem(n, 2, smooth_seed=2000 + q, rhs_seed=3000 + q, nrhs=4) for q, n in enumerate(sizes)]
    probs = [(T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)) for pb in pbs]
    F = T(np.vstack([pb.f for pb in pbs]).T).t()
    dofs = sum(pb.N for pb in pbs)

    def batched(precision):
        fb = P.Factorization.batched(probs, 0, 1e-6, precision=precision)
        u, its, rel = fb.solve_refined(F, tol=TOL)
        fb.close()
        return its, rel

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    for _ in range(args.warmup):
        batched("fp32")
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = H.hif_kernel_launches()
    ts = []
    for _ in range(args.steps):
        t, (its, rel) = timed(lambda: batched("fp32"))
        ts.append(t)
    launches = (H.hif_kernel_launches() - l0) // max(args.steps, 1)
    clocks = sampler.stop()
    t32 = max_over_ranks(sum(ts) / len(ts), world, dev)
    t64, (its64, rel64) = timed(lambda: batched("fp64"))

    def sequential():
        worst, its_max = 0.0, 0
        for q, pb in enumerate(pbs):
            fi = P.Factorization(*probs[q], 0, 1e-6, precision="fp64")
            u, it, r = fi.solve_refined(T(pb.f.T).t(), tol=TOL)
            worst, its_max = max(worst, r), max(its_max, it)
            fi.close()
        return its_max, worst
    tseq, (itss, rels) = timed(sequential) if not args.no_sequential else (float("nan"), (None, None))
    if rank == 0:
        line = {
            "metric": "batched factor + solve DOF/s to rel. residual 1e-10 (independent problems, one handle)",
            "value": job_value(dofs * 4, world, t32), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 factor; residual bf16 digits, exact int sums", "data": "synthetic",
            "config": {"workload": (f"batched: {args.problems} independent 2D second-kind volume IEs, n drawn from "
                                    f"{{32,48,...,256}} (seed 1004), b=c=1+0.5*phi_p (seed 2000+p), eps 1e-6, 4 Gaussian RHS "
                                    f"each (seed 3000+p), refined to "
                                    f"{TOL:g}"), "problems": args.problems, "dofs": dofs, "nrhs": 4,
                       "parallelism": f"replicas x{world}"},
            "refine_iters": its, "relres": rel, "gpu_launches": int(launches), "clocks": clocks,
            "batched_fp64": {"seconds": t64, "value": dofs * 4 / t64, "iters": its64, "relres": rel64},
            "sequential_fp64": {"seconds": tseq, "value": dofs * 4 / tseq if tseq == tseq else None,
                                "iters": itss, "relres": rels},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_examples(args):
    """The rows of the paper's Example 1 and Example 2 tables (Sec. 5): the
    volume IE with a = 0 (Example 1, first kind) or a = 1 (Example 2, second
    kind), b = c = 1, on the n x n grid, factored in FP64 by RSF (``rsf``:
    fractional levels off, Algorithm 3.1), by HIF-IE without the Sec. 4.4
    modifications (``hif``, the paper's hifie2) and with them (``hifx``,
    hifie2x).  One JSON line per (method, eps) with |s_L|, t_f, m_f, t_a/s
    (one apply and one solve, 1 RHS), e_a and e_s (power iteration from a
    uniform start, stopped at 1e-2) and n_i (GMRES with F^{-1} as right
    preconditioner to 1e-12 from a uniform random right-hand side)."""
    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    dev = torch.device(f"cuda:{local}")
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev)
    example = 2 if args.workload == "example2" else 1
    pb = hi.volume_problem(args.n, 2, a_value=0.0 if example == 1 else 1.0)
    ins = [T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)]
    v0 = T(hi.uniform_vector(pb.N, 3))
    f = T(hi.uniform_vector(pb.N, 5))

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    # warm-up: library load, tensor-core table digits, graph capture
    w = P.Factorization(*ins, 0, 1e-3)
    w.apply(f)
    w.matvec(f)
    w.close()
    methods = args.methods or ("hif,rsf" if example == 1 else "hif,hifx,rsf")
    for method in methods.split(","):
        for eps in [float(e) for e in args.eps_list.split(",")]:
            t_f, fac = timed(lambda: P.Factorization(*ins, 0, eps, fractional=method != "rsf",
                                                     second_kind=method == "hifx"))
            fac.apply(f)
            fac.solve(f)
            t_a = min(timed(lambda: fac.apply(f))[0] for _ in range(3))
            t_s = min(timed(lambda: fac.solve(f))[0] for _ in range(3))
            t_e, est = timed(lambda: fac.error_estimates(v0))
            t_g, (u, n_i, rel) = timed(lambda: fac.solve_refined(f, tol=1e-12, method="gmres"))
            st = fac.stats()
            line = {
                "metric": f"Example {example} table row ({'first' if example == 1 else 'second'}-kind volume IE, "
                          "Sec. 5)", "method": method,
                "n": args.n, "N": pb.N, "eps": eps, "second_kind_mode": method == "hifx", "dtype": "f64",
                "data": "synthetic",
                "s_L": st["top_size"], "t_f": t_f, "m_f_gb": st["factor_bytes"] / 1e9, "t_a": t_a, "t_s": t_s,
                "e_a": est["e_a"], "e_s": est["e_s"], "power_iters": est["iters"], "t_estimates": t_e,
                "n_i": n_i, "gmres_relres": rel, "t_gmres": t_g, "levels": st["levels"],
                "sublevels": st["sublevels"],
            }
            print(json.dumps(line), flush=True)
            fac.close()


def run_example3(args):
    """Rows of the paper's Example 3 tables (Sec. 5): the Lippmann-Schwinger
    equation for Helmholtz scattering, kernel (i/4) H_0^(1)(k r), a = 1,
    b = c = k sqrt(omega) with the Gaussian bump omega = exp(-32 |x - x0|^2),
    kappa = n / 32 wavelengths across the square (32 DOFs per wavelength),
    factored in FP64 by HIF-IE with and without the Sec. 4.4 modifications
    (hifx, hif) and by RSF.  One JSON line per (method, eps): |s_L|, t_f, m_f,
    t_a/s, e_a, e_s (power iteration on the complex operator's real
    embedding, from a uniform start, stopped at 1e-2) and n_i (GMRES with
    F^{-1} as right preconditioner to 1e-12 from a complex Gaussian
    right-hand side)."""
    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    dev = torch.device(f"cuda:{local}")
    n = args.n if args.n != 1024 else 128
    pb = hi.helmholtz_problem(n, n / 32.0)
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), device=dev)
    ins = [T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)]
    v0 = T(hi.uniform_vector(2 * pb.N, 3))
    f = T(pb.f[:, 0])

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    w = P.Factorization(*ins, 2, 1e-3, wavenumber=pb.k)
    w.apply(f)
    w.close()
    methods = args.methods or "hif,hifx,rsf"
    for method in methods.split(","):
        for eps in [float(e) for e in args.eps_list.split(",")]:
            t_f, fac = timed(lambda: P.Factorization(*ins, 2, eps, wavenumber=pb.k, fractional=method != "rsf",
                                                     second_kind=method == "hifx"))
            fac.apply(f)
            fac.solve(f)
            t_a = min(timed(lambda: fac.apply(f))[0] for _ in range(3))
            t_s = min(timed(lambda: fac.solve(f))[0] for _ in range(3))
            t_e, est = timed(lambda: fac.error_estimates(v0))
            t_g, (u, n_i, rel) = timed(lambda: fac.solve_refined(f, tol=1e-12, method="gmres"))
            st = fac.stats()
            line = {
                "metric": "Example 3 table row (Lippmann-Schwinger, Helmholtz, Sec. 5)", "method": method,
                "n": n, "N": pb.N, "kappa": n / 32.0, "k": pb.k, "eps": eps, "second_kind_mode": method == "hifx",
                "dtype": "f64 (complex through the real 2x2 embedding)", "data": "synthetic",
                "s_L_real_dofs": st["top_size"], "t_f": t_f, "m_f_gb": st["factor_bytes"] / 1e9, "t_a": t_a,
                "t_s": t_s, "e_a": est["e_a"], "e_s": est["e_s"], "power_iters": est["iters"], "t_estimates": t_e,
                "n_i": n_i, "gmres_relres": rel, "t_gmres": t_g, "levels": st["levels"],
                "sublevels": st["sublevels"],
            }
            print(json.dumps(line), flush=True)
            fac.close()


def run_adjoint(args):
    """The adjoint workload: 2D second-kind IE on the n = 256 grid (N = 65,536),
    b = c = 1 + 0.5 phi (seed 1005), eps = 1e-9, FP64 factorization; loss
    0.5 |u - u*|^2 with u* Gaussian (seed 1007); one step = the forward refined
    solve (to 1e-14) and the backward pass (transposed refined solve and the
    coefficient gradients) through HIFSolve, after the factorization, which
    is timed separately."""
    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    from paper_1307_2666_gb300 import hif as H
    dev = torch.device(f"cuda:{local}")
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev)
    n, eps, tol = 256, 1e-9, 1e-14
    pb = hi.volume_problem(n, 2, smooth_seed=1005, rhs_seed=1006)
    ustar = T(hi.gaussian_rhs(pb.N, 1, 1007)[:, 0])
    ins = [T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)]

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    t_f, fac = timed(lambda: P.Factorization(*ins, 0, eps))

    def step():
        leaves = [T(pb.f[:, 0]).requires_grad_(True)] + [x.clone().requires_grad_(True) for x in ins[2:]]
        u = P.HIFSolve.apply(*leaves, fac, tol)
        loss = 0.5 * torch.sum((u - ustar) ** 2)
        loss.backward()
        return loss, [x.grad for x in leaves]

    for _ in range(args.warmup):
        step()
    l0 = H.hif_kernel_launches()
    ts = []
    for _ in range(args.steps):
        t, (loss, grads) = timed(step)
        ts.append(t)
    launches = (H.hif_kernel_launches() - l0) // max(args.steps, 1)
    t_fwd, _ = timed(lambda: fac.solve_refined(T(pb.f[:, 0]), tol=tol))
    ms = 1000 * sum(ts) / len(ts)
    line = {"metric": "adjoint: forward + backward steps per second (refined solves to 1e-14, FP64 factor)",
            "value": 1000.0 / ms, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "adjoint: 2D second-kind IE n=256 (N=65,536), b=c=1+0.5*phi (seed 1005), "
                                   "eps=1e-9, FP64, loss 0.5|u-u*|^2, gradients wrt f, a, b, c"},
            "t_factor_s": t_f, "t_forward_s": t_fwd, "loss": float(loss.detach()),
            "grad_norms": {k: float(torch.linalg.norm(g)) for k, g in zip("fabc", grads)},
            "gpu_launches": int(launches)}
    fac.close()
    print(json.dumps(line), flush=True)


def run_grid3d(args):
    """The 3D workload: second-kind volume IE on the unit cube, kernel
    1/(4 pi r), n = 64 (N = 262,144) unless --n is given, b = c = 1 + 0.5 phi
    (seed 1008), 16 Gaussian RHS (seed 1009); for each eps of --eps-list the
    FP32 factorization refined to 1e-10 against the direct sum and, unless
    --no-compare-fp64, the FP64 factorization refined the same way.  One JSON
    line per (precision, eps) with the factor and refined-solve times."""
    import numpy as np
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import hif_inputs as hi
    import paper_1307_2666_gb300 as P
    dev = torch.device(f"cuda:{local}")
    n = args.n if args.n != 1024 else 64
    nrhs = args.nrhs if args.nrhs != 8 else 16
    pb = hi.volume_problem(n, 3, smooth_seed=1008, rhs_seed=1009, nrhs=nrhs)
    T = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device=dev)
    ins = [T(pb.points), T(pb.weights), T(pb.a), T(pb.b), T(pb.c)]
    F = T(pb.f.T).t()

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, out

    w = P.Factorization(*ins, 1, 1e-1, proxy_dirs=pb.proxy, precision="fp32")
    w.close()
    precs = ["fp32", "fp64"] if args.compare_fp64 else ["fp32"]
    for eps in [float(e) for e in args.eps_list.split(",")]:
        for prec in precs:
            t_f, fac = timed(lambda: P.Factorization(*ins, 1, eps, proxy_dirs=pb.proxy, precision=prec))
            t_s, (u, its, rel) = timed(lambda: fac.solve_refined(F, tol=TOL, method="ir"))
            st = fac.stats()
            line = {"metric": "3D second-kind volume IE: factor + refined solve to 1e-10", "precision": prec,
                    "n": n, "N": pb.N, "nrhs": nrhs, "eps": eps, "data": "synthetic",
                    "config": {"workload": f"3D second-kind volume IE, unit cube, n={n} (N={pb.N}), kernel "
                                           f"1/(4 pi r), a=1, b=c=1+0.5*phi (seed 1008), {nrhs} Gaussian RHS "
                                           f"(seed 1009), eps={eps:g}, {prec.upper()} factorization + iterative "
                                           "refinement to 1e-10 against the direct sum"},
                    "t_factor_s": t_f, "t_solve_s": t_s, "refine_iters": its, "relres": rel,
                    "dofs_per_s": pb.N * nrhs / (t_f + t_s), "top_size": st["top_size"],
                    "factor_bytes": st["factor_bytes"], "levels": st["levels"], "sublevels": st["sublevels"]}
            print(json.dumps(line), flush=True)
            fac.close()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    sample = None
    for _ in range(args.warmup):
        run_oracle_subprocess()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = run_oracle_subprocess()
        vals.append(s["seconds"])
        sample = s
    t = time.perf_counter() - t0
    value = sample["N"] * args.steps / sum(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(vals) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args.n, args.nrhs, args.eps), parallelism="host cores x1"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": t}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--nrhs", type=int, default=8)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["grid", "grid3d", "batched", "example1", "example2", "example3", "adjoint"],
                    default="grid",
                    help="grid: the n x n bench workload (default); batched: independent problems in one handle; "
                         "example1 / example2: the paper's first- / second-kind table rows (RSF and HIF-IE); "
                         "example3: the Helmholtz (Lippmann-Schwinger) table rows, n = 128 unless --n is given; "
                         "grid3d: the 3D n = 64 workload (16 RHS) at each eps of --eps-list, FP32 and FP64")
    ap.add_argument("--methods", default=None,
                    help="example workloads: any of rsf, hif (hifie2), hifx (hifie2x); default hif,rsf for "
                         "example1 and hif,hifx,rsf for example2")
    ap.add_argument("--eps-list", default="1e-3,1e-6,1e-9", help="example workloads: tolerances")
    ap.add_argument("--problems", type=int, default=256, help="batched workload: number of problems")
    ap.add_argument("--no-sequential", action="store_true", help="batched workload: skip the one-by-one leg")
    ap.add_argument("--oracle-sample-json", type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample_json is not None:
        print(json.dumps(oracle_sample(args.oracle_sample_json)))
        return
    if args.warmup < 3 and args.impl == "gpu":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload in ("example1", "example2"):
        run_examples(args)
    elif args.workload == "example3":
        run_example3(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "grid3d":
        run_grid3d(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
