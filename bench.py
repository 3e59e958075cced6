#!/usr/bin/env python3
"""Benchmark of the spectral multigrid PCG solve on one GB300 per rank.

Metric: solve DOF/s to rtol 1e-8 (mixed vs FP64 form) and the V-cycle's HBM
fraction of peak.  A step is one complete PCG solve (to ||b - A x|| <=
1e-8 ||b||) of the default workload: a 128^3 high-contrast inclusion field
(background 1, 200 random spheres and 20 full-length 2x2 channels at 1e6),
8^3 elements, 4 levels, 6 eigenvectors per local problem.  Set-up is done
once before timing and reported separately.  Inputs are synthetic and
seeded; they are resident in HBM when the timed region starts, and L2 is
flushed (256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload batched [--steps K] [--warmup W]
  python bench.py --workload layered [--steps K] [--warmup W]
  python bench.py --workload scale [--steps K] [--warmup W] [--hierarchy stated]
  python bench.py --workload strategy2 [--steps K] [--warmup W]
  python bench.py --workload network [--steps K] [--warmup W]
  python bench.py --workload impes [--steps K] [--warmup W]

The default line also carries ``batched_rhs``: the same workload with 16
zero-mean random right-hand sides solved in one call (one launch sequence for
all 16, rhs-minor CTA order).  ``--workload batched`` measures the batched
workload instead: 8 lognormal realisations (sigma_logk 2 + 2i/7, correlation
length 0.1) on 64^3, 64^3, 96^3, 96^3, 128^3, 128^3, 192^3, 192^3 grids with
16 random zero-mean right-hand sides each, all solved by one
msmg_solve_batched call (one stream per problem, CUDA graphs).
``--workload layered`` measures the learned warm start: a 512^3 layered field
with sinuous channels (85 layers, contrast 1e6-1e8, seed 100), 8^3 elements,
6 levels, 12 eigenvectors per local problem; the network is trained first on
eigenpairs the library computes for held-out 128^3 fields of the same kind
(seeds 101-110); set-up is timed cold and warm-started, then the mixed solve.
``--workload scale`` is the single-GPU limit: a 1024^3 lognormal field (contrast
1e6), 8^3 elements, 7 levels, 4 eigenvectors per local problem, mixed form.

With N > 1 (torchrun) every rank solves its own replica of the workload (the
solve is not sharded across GPUs): weak scaling, no data-path collective;
value = DOF solved by all ranks / max time.
``--impl reference`` times the FP64 CPU oracle (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve DOF/s to rtol 1e-8 (mixed vs FP64 form); V-cycle HBM % of peak"
WORKLOAD = ("128^3 unit-cube inclusion field: background 1, 200 spheres (radius 1.5h-6h) and 20 axis-aligned "
            "2x2-cell channels at 1e6 (seed 1); corner source/sink; 8^3 elements, 4 levels (ratio 2), "
            "6 eigenvectors per local problem; PCG rtol 1e-8")
N_GRID = 128
BLOCK = (8, 8, 8)
N_LEVELS = 4
N_EIG = [6, 6, 6]
RATIO = [(2, 2, 2), (2, 2, 2)]
RTOL = 1e-8
BATCH_RHS = 16
C3_GRIDS = [64, 64, 96, 96, 128, 128, 192, 192]   # fields.LOGNORMAL_BATCH_GRIDS
C3_WORKLOAD = ("8 lognormal realisations (sigma_logk = 2 + 2i/7, i = 0..7, exponential covariance, correlation "
               "length 0.1, seeds 10..17) on 64^3, 64^3, 96^3, 96^3, 128^3, 128^3, 192^3, 192^3 unit-cube grids, "
               "16 iid N(0,1) zero-mean right-hand sides each; 8^3 elements, 4 levels (ratio 2), 4 eigenvectors "
               "per local problem; one msmg_solve_batched call; PCG rtol 1e-8")


def field():
    import fields
    return fields.inclusions(N_GRID, seed=1, n_spheres=200, n_channels=20, k_hi=1e6)


def rhs(shape):
    import fields
    return fields.rhs_corners(shape)


# Algorithmic bytes per fine cell and launch of each fine-level kernel of one PCG
# iteration (halos excluded), by form; L = eigenvectors per element, v = bytes of
# a V-cycle value (4 mixed, 8 FP64).
#   pre:      x, r read+write, p, q read (FP64); r copy and u written (v); T (3), 1/d read (v)
#   restrict: r copy, u (v); T (3) (v); basis (L values, v)
#   prolong:  (separate variant) basis (L values, v); u read and written (v)
#   post:     r copy (mixed form only; the FP64 form reads r once for both), u (v);
#             T (3), 1/d (v); the basis (L values, v) only in the fused variant,
#             where the prolongation runs inside it; r read (FP64); q read (FP64,
#             flexible beta only); z written (FP64)
#   pmatvec:  z, p_old read, p_new, q written (FP64); T (3) and the diagonal D (FP64)
# With R right-hand sides in one launch the coefficients (T, 1/d, D, basis) are read
# once for all R: bytes per cell and right-hand side.  fused: the variant the
# autotuner picked (Solver.info["tuning"][0] for one right-hand side, [1] for R).
def kernel_bytes(form: str, L: int, R: int = 1, fused: bool = False) -> dict:
    v = 4 if form == "mixed" else 8
    flex = 8 if form == "mixed" else 0
    basis = L * v / R
    return {"pre": 48 + 2 * v + 4 * v / R, "restrict": 2 * v + (3 * v) / R + basis,
            "prolong": 0.0 if fused else basis + 2 * v,
            "post": (2 * v if form == "mixed" else v) + (4 * v) / R + (basis if fused else 0.0) + 8 + flex + 8,
            "pmatvec": 32 + 32 / R}


VCYCLE_FINE = ("pre", "restrict", "prolong", "post")

# Algorithmic FP64 flops per fine cell and launch in the mixed form (FMA = 2):
#   pre      x += alpha p, r -= alpha q, r.r                          3 FMA
#   post     r.z and z.q (flexible beta)                              2 FMA
#   pmatvec  p = z + beta p_old, (A p)_c = D_c p_c - 6 T p_nb, p.q   1 MUL + 8 FMA
# (restrict and prolong run in FP32.)  GB300 issues FP64 at 2 FMA per clock
# per SM, so these are the kernels whose FP64 rate can bind before HBM does.
FP64_FLOPS_MIXED = {"pre": 6, "restrict": 0, "prolong": 0, "post": 4, "pmatvec": 17}
N_SMS = 152


def fp64_peak_gflops(sm_mhz: float) -> float:
    """FP64 peak from unit counts and clock: 152 SMs x 2 FMA/clock x 2 flops."""
    return N_SMS * 2 * 2 * sm_mhz * 1e-3


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel: str, fused: bool):
    """Per-launch DRAM bytes of ``kernel`` from the committed ncu summary, if it
    was captured on the current source of the kernel file and in the same
    prolongation variant."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        src = os.path.join(ROOT, "paper_2403_19342_gb300", "csrc", rec["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        ent = rec["kernels"].get(kernel)
        variant = "fused" if fused else "separate"
        if ent and rec.get("source_sha") == sha and rec.get("prolongation") == variant:
            return ent["dram_bytes_per_launch_full_size"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, units_per_rank: float, ms_per_step_local: float) -> tuple[float, float]:
    """Whole-job throughput of N independent replicas (weak scaling): the units all
    ranks processed divided by the slowest rank's time; returns (value, max ms)."""
    ms = max_over_ranks(world, ms_per_step_local)
    return world * units_per_rank / (ms * 1e-3), ms


# ------------------------------------------------------------------ reference arm / CPU baseline
CROP = 64


def oracle_sample(steps: int = 1, keep: bool = False, warmup: int = 0):
    """The FP64 oracle as it stands on a bounded sample of the workload: the
    64^3 corner crop of the same field, same hierarchy parameters, same RHS
    pattern; setup excluded from the metric.  With keep, the record also holds
    the crop, its right-hand side and the oracle's hierarchy."""
    import oracle
    kappa = field()[:CROP, :CROP, :CROP].copy()
    f = rhs(kappa.shape).ravel()
    opts = oracle.Options(n_levels=N_LEVELS, block=BLOCK, ratio=RATIO, n_eig=N_EIG, nu=[1] * (N_LEVELS - 1))
    t0 = time.perf_counter()
    H = oracle.setup(kappa, (1.0 / N_GRID,) * 3, opts)
    t1 = time.perf_counter()
    for _ in range(warmup):                     # untimed
        oracle.solve(H, f, rtol=RTOL)
    times, its = [], []
    for _ in range(steps):
        s0 = time.perf_counter()
        res = oracle.solve(H, f, rtol=RTOL)
        times.append(time.perf_counter() - s0)
        its.append(res.iterations)
    n = kappa.size
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rec = {"value": n / float(np.mean(times)), "unit": "DOF/s", "cores": cores, "kind": "oracle",
           "sample": f"{CROP}^3 corner crop of the same field and hierarchy, full PCG solve to rtol 1e-8 "
                     f"({its[0]} iterations); oracle setup {t1 - t0:.1f} s excluded like the GPU setup",
           "setup_s": t1 - t0, "solve_s": float(np.mean(times)), "iterations": its[0]}
    if keep:
        rec.update(kappa=kappa, f=f, H=H)
    return rec


def error_vs_oracle(pkg, rec) -> dict:
    """Error of each GPU form against the FP64 oracle, stated per result: the 64^3
    crop solved by the GPU (its own bases, rtol 1e-8) and by the oracle to rtol
    1e-12 (the reference solution; both zero-mean)."""
    import oracle
    import torch
    kappa, f, H = rec["kappa"], rec["f"], rec["H"]
    ref = None
    for tol in (1e-11, 1e-10):          # tighter solves meet rounding (p^T A p <= 0) at contrast 1e6
        try:
            ref = oracle.solve(H, f, rtol=tol)
            break
        except FloatingPointError:
            continue
    if ref is None:
        return {"unavailable": "the oracle's reference solve broke down at rtol 1e-10"}
    out = {"sample": f"{CROP}^3 corner crop, hierarchy of the workload; oracle solution to rtol {tol:g} "
                     f"({ref.iterations} iterations); GPU solves to rtol 1e-8 with their own bases",
           "metric": "||x_gpu - x_oracle||_2 / ||x_oracle||_2"}
    for form, prec in (("fp64", pkg.FP64), ("mixed", pkg.MIXED)):
        S = pkg.Solver(torch.tensor(kappa, device="cuda"),
                       pkg.Options(n_levels=N_LEVELS, block=BLOCK, ratio=RATIO, n_eig=N_EIG, precision=prec,
                                   eig_tol=1e-8), h=(1.0 / N_GRID,) * 3)
        x, info, _ = S.solve(torch.tensor(f.reshape(kappa.shape), device="cuda"), rtol=RTOL)
        xe = x.cpu().numpy().ravel()
        out[form] = {"error": float(np.linalg.norm(xe - ref.x) / np.linalg.norm(ref.x)),
                     "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"]}
        S.close()
    return out


def two_grid_record(pkg, kappa, f_dev, args, world, flush, stream, forms) -> dict:
    """The exact two-grid preconditioner P_TG (Eq. (B_TG)) on the same workload: the
    level-2 system solved by the inner PCG to 1e-10 every outer iteration, against
    the V-cycle (P_ITG) of the main measurement."""
    import torch
    out = {"inner_rtol": 1e-10}
    for form, prec in (("fp64", pkg.FP64), ("mixed", pkg.MIXED)):
        S = pkg.Solver(kappa, pkg.Options(n_levels=N_LEVELS, block=BLOCK, ratio=RATIO, n_eig=N_EIG, precision=prec,
                                          eig_tol=1e-8, two_grid=True, inner_rtol=1e-10, inner_max_iter=500))
        x = torch.zeros_like(f_dev)
        pkg.msmg_solve(S.ctx, f_dev, x, RTOL, 1000, 0)
        torch.cuda.synchronize()
        ms, info = [], None
        for k in range(max(1, min(args.steps, 2))):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st, info = pkg.msmg_solve(S.ctx, f_dev, x, RTOL, 1000, 0)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        step = max_over_ranks(world, float(np.mean(ms)))
        out[form] = {"ms_per_step": step, "iterations": info[0]["iterations"],
                     "inner_iterations": info[0]["inner_iterations"],
                     "true_rel_residual": info[0]["true_rel_residual"],
                     "p_itg_ms_per_step": forms[form]["ms_per_step"], "p_itg_iterations": forms[form]["iterations"]}
        S.close()
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    # each step a bounded sample (the 64^3 crop); at most 3 timed and 3 untimed
    # solves keep the run within a few minutes of host time
    steps = max(1, min(args.steps, 3))
    warm = max(0, min(args.warmup, 3))
    rec = oracle_sample(steps, warmup=warm)
    line = {"impl": "reference", "metric": METRIC, "value": rec["value"], "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": rec["solve_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": rec["sample"]},
            "cpu_baseline": {k: rec[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": rec["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def batched_rhs(pkg, S, shape, n, args, world, flush, stream):
    """The same workload with BATCH_RHS zero-mean random right-hand sides in one
    msmg_solve call (mixed form)."""
    import torch
    import fields
    F = torch.tensor(fields.rhs_random(shape, BATCH_RHS, seed=2024), device=stream.device)
    X = torch.zeros_like(F)
    for _ in range(max(1, args.warmup)):
        pkg.msmg_solve(S.ctx, F, X, RTOL, 1000, 0)
    torch.cuda.synchronize()
    barrier(world)
    ms = []
    infos = None
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, infos = pkg.msmg_solve(S.ctx, F, X, RTOL, 1000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    step = max_over_ranks(world, float(np.mean(ms)))
    its = [i["iterations"] for i in infos]
    kt = S.time_kernels(reps=5, n_rhs=BATCH_RHS)
    kb = kernel_bytes("mixed", N_EIG[0], BATCH_RHS, fused=S.info["tuning"][1] == 1)
    vc = sum(kb[k] for k in VCYCLE_FINE) * n * BATCH_RHS
    peak, _ = load_peaks()
    return {"n_rhs": BATCH_RHS, "value": world * n * BATCH_RHS / (step * 1e-3), "unit": "DOF/s",
            "ms_per_step": step, "iterations_min": min(its), "iterations_max": max(its),
            "true_rel_residual_max": max(i["true_rel_residual"] for i in infos),
            "converged": all(i["converged"] for i in infos), "kernel_ms": kt,
            "vcycle_hbm_frac": vc / (kt["vcycle"] * 1e-3) / 1e9 / peak,
            "gpu_launches": int(infos[0]["kernel_launches"])}


def run_gpu(args, world, rank, local):
    import torch
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kappa_np = field()
    shape = kappa_np.shape
    n = int(np.prod(shape))
    kappa = torch.tensor(kappa_np, device=dev)
    f_np = rhs(shape)
    f_dev = torch.tensor(f_np, device=dev)
    x_dev = torch.zeros_like(f_dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    forms = {}
    kernel_times = {}
    sampler = ClockSampler(local)
    launches = 0
    batched = None
    for form, prec in (("fp64", pkg.FP64), ("mixed", pkg.MIXED)):
        opts = pkg.Options(n_levels=N_LEVELS, block=BLOCK, ratio=RATIO, n_eig=N_EIG, precision=prec, eig_tol=1e-8,
                           autotune=True)
        S = pkg.Solver(kappa, opts, n_rhs=BATCH_RHS if form == "mixed" else 1, tuning_cache=args.tuning_cache)
        info0 = S.info
        for _ in range(args.warmup):
            pkg.msmg_solve(S.ctx, f_dev, x_dev, RTOL, 1000, 0)
        torch.cuda.synchronize()
        barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if form == "mixed":
            sampler.start()
        torch.cuda.synchronize()
        infos = []
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            st, info = pkg.msmg_solve(S.ctx, f_dev, x_dev, RTOL, 1000, 0)
            ev[k][1].record(stream)
            infos.append(info[0])
        torch.cuda.synchronize()
        barrier(world)
        if form == "mixed":
            clocks = sampler.stop()
        ms = [a.elapsed_time(b) for a, b in ev]
        ms_step = max_over_ranks(world, float(np.mean(ms)))
        inf = infos[-1]
        if form == "mixed":
            launches = int(sum(i["kernel_launches"] for i in infos))
        forms[form] = {"value": world * n / (ms_step * 1e-3), "unit": "DOF/s", "ms_per_step": ms_step,
                       "tuning": info0["tuning"],
                       "iterations": inf["iterations"], "true_rel_residual": inf["true_rel_residual"],
                       "converged": bool(inf["converged"]), "setup_ms": info0["setup_ms"],
                       "eig_ms": info0["eig_ms"], "eig_residual_max": info0["eig_residual_max"],
                       "eig_iterations_max": info0["eig_iterations_max"]}
        kernel_times[form] = S.time_kernels(reps=10)
        if form == "mixed":
            # end to end through the C-ABI with host buffers (pinned), copies inside the timed region
            f_host = torch.tensor(f_np).pin_memory()
            x_host = torch.zeros_like(f_host).pin_memory()
            pkg.msmg_solve(S.ctx, f_host, x_host, RTOL, 1000, pkg.FLAG_HOST_IO)
            torch.cuda.synchronize()
            e2e_ms = []
            for k in range(args.steps):
                flush.fill_(float(k))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pkg.msmg_solve(S.ctx, f_host, x_host, RTOL, 1000, pkg.FLAG_HOST_IO)
                b.record(stream)
                torch.cuda.synchronize()
                e2e_ms.append(a.elapsed_time(b))
            e2e_step = max_over_ranks(world, float(np.mean(e2e_ms)))
            e2e = {"value": world * n / (e2e_step * 1e-3), "unit": "DOF/s", "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_step}
            batched = batched_rhs(pkg, S, shape, n, args, world, flush, stream)
        S.close()
        del S
    # roofline of the dominant fine-level kernel of the mixed V-cycle
    peak, peak_kind = load_peaks()
    L = N_EIG[0]
    kb = kernel_bytes("mixed", L, fused=forms["mixed"]["tuning"][0] == 1)
    kt = kernel_times["mixed"]
    fine = {k: kt[k] for k in ("pre", "restrict", "prolong", "post", "pmatvec") if kb[k] > 0}
    dom = max(fine, key=fine.get)
    # each fine kernel against both of its ceilings: HBM bandwidth (measured copy
    # peak) and the FP64 rate (from unit counts at the maximum SM clock)
    f64_peak = fp64_peak_gflops(float(clocks.get("sm_max_mhz") or 2070.0))
    per_kernel = {}
    for k, t in fine.items():
        gbs = kb[k] * n / (t * 1e-3) / 1e9
        gfl = FP64_FLOPS_MIXED[k] * n / (t * 1e-3) / 1e9
        per_kernel[k] = {"ms": t, "hbm_gbs": gbs, "hbm_frac": gbs / peak, "fp64_gflops": gfl,
                         "fp64_frac": gfl / f64_peak}
    pk = per_kernel[dom]
    traffic = traffic_record(dom, forms["mixed"]["tuning"][0] == 1)
    if pk["fp64_frac"] > pk["hbm_frac"]:
        roofline = {"bound": "alu", "kernel": dom, "achieved": pk["fp64_gflops"] * 1e-3,
                    "peak": f64_peak * 1e-3, "unit": "TFLOP/s", "frac": pk["fp64_frac"], "traffic": traffic,
                    "peak_source": "derived: FP64, 152 SMs x 2 FMA/clock x 2 flops x max SM clock",
                    "algorithmic_flops_per_launch": FP64_FLOPS_MIXED[dom] * n,
                    "hbm": {"achieved": pk["hbm_gbs"], "peak": peak, "unit": "GB/s", "frac": pk["hbm_frac"],
                            "peak_source": peak_kind},
                    "algorithmic_bytes_per_launch": kb[dom] * n, "avg_launch_ms": kt[dom]}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": pk["hbm_gbs"], "peak": peak, "unit": "GB/s",
                    "frac": pk["hbm_frac"], "traffic": traffic, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": kb[dom] * n, "avg_launch_ms": kt[dom]}
    roofline["per_kernel"] = per_kernel
    vc_bytes = sum(kb[k] for k in VCYCLE_FINE) * n
    vc_frac = vc_bytes / (kt["vcycle"] * 1e-3) / 1e9 / peak
    kb64 = kernel_bytes("fp64", L, fused=forms["fp64"]["tuning"][0] == 1)
    vc64 = sum(kb64[k] for k in VCYCLE_FINE) * n / (kernel_times["fp64"]["vcycle"] * 1e-3) / 1e9 / peak
    line = {"metric": METRIC, "value": forms["mixed"]["value"], "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms["mixed"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "flushed before each step (256 MiB write); working set > L2",
                       "form": "mixed: FP32 fine V-cycle and bases, FP64 coarse levels and outer PCG",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "forms": forms,
            "vcycle_hbm_frac": {"mixed": vc_frac, "fp64": vc64, "peak_gbs": peak},
            "kernel_ms": kernel_times,
            "batched_rhs": batched,
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks}
    line["two_grid"] = two_grid_record(pkg, kappa, f_dev, args, world, flush, stream, forms)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rec = oracle_sample(1, keep=True)
        line["cpu_baseline"] = {k: rec[k] for k in ("value", "unit", "cores", "kind", "sample")}
        line["error_vs_oracle"] = error_vs_oracle(pkg, rec)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batched(args, world, rank, local):
    """The batched workload: 8 problems of uneven size, 16 right-hand sides each,
    one msmg_solve_batched call per step (mixed form)."""
    import torch
    import fields
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    solvers, F, X, Fh, Xh = [], [], [], [], []
    setup_ms, eig_ms, total = [], [], 0
    for N, (kappa, f) in zip(C3_GRIDS, fields.lognormal_batch(BATCH_RHS, C3_GRIDS, device="cuda")):
        opts = pkg.Options(n_levels=4, block=(8, 8, 8), ratio=[(2, 2, 2), (2, 2, 2)], n_eig=[4, 4, 4],
                           precision=pkg.MIXED, eig_tol=1e-8, autotune=True)
        S = pkg.Solver(torch.tensor(kappa, device=dev), opts, n_rhs=BATCH_RHS)
        solvers.append(S)
        setup_ms.append(S.info["setup_ms"])
        eig_ms.append(S.info["eig_ms"])
        F.append(torch.tensor(f, device=dev))
        X.append(torch.zeros_like(F[-1]))
        Fh.append(torch.tensor(f).pin_memory())
        Xh.append(torch.zeros_like(Fh[-1]).pin_memory())
        total += N ** 3 * BATCH_RHS
    ctxs = [S.ctx for S in solvers]
    for _ in range(args.warmup):
        pkg.msmg_solve_batched(ctxs, F, X, RTOL, 2000, 0)
    torch.cuda.synchronize()
    barrier(world)
    sampler = ClockSampler(local)
    sampler.start()
    ms, infos = [], None
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, infos = pkg.msmg_solve_batched(ctxs, F, X, RTOL, 2000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    clocks = sampler.stop()
    step = max_over_ranks(world, float(np.mean(ms)))
    # end to end with host buffers (copies inside the call)
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pkg.msmg_solve_batched(ctxs, Fh, Xh, RTOL, 2000, pkg.FLAG_HOST_IO)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_step = max_over_ranks(world, float(np.mean(e2e_ms)))
    # the same problems solved one after another (one call each): what the batched
    # call's concurrency across problems gains
    seq_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for S, f, x in zip(solvers, F, X):
            pkg.msmg_solve_batched([S.ctx], [f], [x], RTOL, 2000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        seq_ms.append(a.elapsed_time(b))
    seq_step = float(np.mean(seq_ms))
    per = []
    for N, inf in zip(C3_GRIDS, infos):
        its = [i["iterations"] for i in inf]
        per.append({"grid": N, "iterations_min": min(its), "iterations_max": max(its),
                    "true_rel_residual_max": max(i["true_rel_residual"] for i in inf),
                    "converged": all(i["converged"] for i in inf)})
    launches = int(sum(inf[0]["kernel_launches"] * ((BATCH_RHS + solvers[j].max_batch_rhs - 1)
                                                   // solvers[j].max_batch_rhs)
                       for j, inf in enumerate(infos)))
    line = {"metric": METRIC, "value": world * total / (step * 1e-3), "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": C3_WORKLOAD, "form": "mixed", "n_rhs_per_problem": BATCH_RHS,
                       "l2": "flushed before each step (256 MiB write); working set > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "problems": per, "setup_ms": setup_ms, "eig_ms": eig_ms,
            "sequential": {"ms_per_step": seq_step, "value": total / (seq_step * 1e-3),
                           "note": "the same problems, one msmg_solve_batched call each, back to back"},
            "e2e": {"value": world * total / (e2e_step * 1e-3), "unit": "DOF/s",
                    "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 8 * total, "ms_per_step": e2e_step},
            "gpu_launches": launches, "clocks": clocks}
    for S in solvers:
        S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


LAYERED_N = 512
LAYERED_WORKLOAD = ("512^3 layered field: 85 z-layers of laterally upsampled 60x220 lognormal lattices, sinuous "
                    "binary channels in 50 layers, contrast U(1e6, 1e8) (seed 100); corner source/sink; 8^3 "
                    "elements, 6 levels (ratio 2), 12 eigenvectors per local problem; PCG rtol 1e-8; learned "
                    "warm start trained on 128^3 fields of the same kind (seeds 101-110)")


def train_warm_start(pkg, torch, fields, L, n_fields=10, N=128, steps=6000, hidden=(1024, 1024)):
    """Train the warm-start network on eigenpairs the library computes for held-out
    fields; returns (net, record)."""
    opts = dict(n_levels=4, block=(8, 8, 8), ratio=[(2, 2, 2)] * 2, n_eig=[L] * 3, precision=pkg.MIXED,
                eig_tol=1e-8)
    t0 = time.perf_counter()
    xs, ys = [], []
    for seed in range(101, 101 + n_fields):
        S = pkg.Solver(torch.tensor(fields.layered_channels((N, N, N), seed=seed), device="cuda"),
                       pkg.Options(**opts))
        x, y = S.learning_data()
        xs.append(x)
        ys.append(y.reshape(y.shape[0], -1))
        S.close()
    X, Y = torch.cat(xs), torch.cat(ys)
    t1 = time.perf_counter()
    net = pkg.WarmStartNet(n_in=512, hidden=hidden, n_vec=L - 1, batch_max=512, seed=7)
    gen = torch.Generator(device="cuda").manual_seed(0)
    loss = None
    for step in range(steps):
        idx = torch.randint(0, X.shape[0], (512,), device="cuda", generator=gen)
        loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr=3e-4 if step < 0.7 * steps else 1e-4)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return net, {"samples": int(X.shape[0]), "eigenpairs": int(X.shape[0]) * (L - 1), "steps": steps,
                 "hidden": list(hidden), "final_batch_loss": loss, "data_s": t1 - t0, "train_s": t2 - t1}


def run_layered(args, world, rank, local):
    import torch
    import fields
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # stated: the configuration as specified (6 eigenvectors, 5 levels: coarsest 3072 unknowns);
    # tuned: 12 eigenvectors and 6 levels (the channels cross many elements: with 6
    # eigenvectors the 128^3 field needs ~1000 PCG iterations, with 12 ~400)
    L, nl = (6, 5) if args.hierarchy == "stated" else (12, 6)
    net, train = train_warm_start(pkg, torch, fields, L)
    kappa = torch.tensor(fields.layered_channels((LAYERED_N,) * 3, seed=100), device=dev)
    n = LAYERED_N ** 3
    base = dict(n_levels=nl, block=(8, 8, 8), ratio=[(2, 2, 2)] * (nl - 2), n_eig=[L] * (nl - 1), precision=pkg.MIXED,
                eig_tol=1e-8, autotune=True)
    recs = {}
    solver = None
    for name, ws in (("cold", None), ("warm", net)):
        S = pkg.Solver(kappa, pkg.Options(**base, warm_start=ws))
        i = S.info
        recs[name] = {"setup_ms": i["setup_ms"], "eig_ms": i["eig_ms"], "eig_iterations_total": i["eig_iterations_total"],
                      "eig_iterations_max": i["eig_iterations_max"], "eig_residual_max": i["eig_residual_max"],
                      "warm_started": i["warm_started"]}
        if name == "warm":
            solver = S
        else:
            S.close()
            del S
    f = torch.tensor(rhs((LAYERED_N,) * 3), device=dev)
    x = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pkg.msmg_solve(solver.ctx, f, x, RTOL, 6000, 0)
    torch.cuda.synchronize()
    ms, info = [], None
    for k in range(args.steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, info = pkg.msmg_solve(solver.ctx, f, x, RTOL, 6000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    step = max_over_ranks(world, float(np.mean(ms)))
    line = {"metric": METRIC, "value": world * n / (step * 1e-3), "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": LAYERED_WORKLOAD.replace("6 levels (ratio 2), 12 eigenvectors",
                                                            f"{nl} levels (ratio 2), {L} eigenvectors"),
                       "hierarchy": args.hierarchy, "form": "mixed, learned warm start",
                       "l2": "flushed before each step (256 MiB write); working set > L2"},
            "iterations": info[0]["iterations"], "true_rel_residual": info[0]["true_rel_residual"],
            "setup": recs, "training": train,
            "setup_speedup": recs["cold"]["setup_ms"] / recs["warm"]["setup_ms"],
            "gpu_launches": int(info[0]["kernel_launches"])}
    solver.close()
    net.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


STRAT2_N = 128
STRAT2_WORKLOAD = ("128^3 layered field of the 512^3 recipe (85 layers, sinuous channels, contrast U(1e6, 1e8), "
                   "seed 100); corner source/sink; 8^3 elements, 3 levels (ratio 2, the paper's three-grid setting), "
                   "12 level-1 eigenvectors; "
                   "level-2 spaces by Strategy 1 (12 or 24 per parent) or Strategy 2 (B_cc among 24 candidates, "
                   "at quantiles of the level-2 local spectra; also B_c among the 12 level-1 candidates); "
                   "PCG rtol 1e-8")


def run_strategy2(args, world, rank, local):
    """Strategy 2 (Section 5) against Strategy 1 on the layered channel field, as
    the paper compares them: L_c fixed, the coarse-coarse dimension chosen by a
    threshold B_cc among 24 candidates (the last run also thresholds level 1),
    mixed form."""
    import torch
    import fields
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = STRAT2_N
    n = N ** 3
    kappa = torch.tensor(fields.layered_channels((N, N, N), seed=100), device=dev)
    f = torch.tensor(rhs((N, N, N)), device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # three levels: with 24 vectors per level-2 parent a third level's local problems would
    # have 8 x 24 unknowns, above the 96 of the shared-memory eigensolver
    base = dict(n_levels=3, block=(8, 8, 8), ratio=[(2, 2, 2)], precision=pkg.MIXED, eig_tol=1e-8, autotune=True)

    def measure(opts, export=False):
        S = pkg.Solver(kappa, pkg.Options(**base, **opts))
        x = torch.zeros_like(f)
        for _ in range(args.warmup):
            pkg.msmg_solve(S.ctx, f, x, RTOL, 3000, 0)
        torch.cuda.synchronize()
        ms, info = [], None
        for k in range(args.steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st, info = pkg.msmg_solve(S.ctx, f, x, RTOL, 3000, 0)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        i0 = S.info
        rec = {"ms_per_step": float(np.mean(ms)), "value": n / (float(np.mean(ms)) * 1e-3),
               "iterations": info[0]["iterations"], "true_rel_residual": info[0]["true_rel_residual"],
               "dims": i0["dims"], "dims_kept": i0["dims_kept"], "setup_ms": i0["setup_ms"], "options": opts}
        lam = (S.export_basis(1)[1].cpu().numpy(), S.export_basis(2)[1].cpu().numpy()) if export else None
        S.close()
        # the FP64 form's count beside it: on this contrast-1e8 field the mixed form's
        # iteration count moves with rounding details (two orders of the same coarse
        # row sums gave 49 and 62 iterations), the FP64 form's does not
        base64 = dict(base, precision=pkg.FP64, autotune=False)
        S = pkg.Solver(kappa, pkg.Options(**base64, **opts))
        x64 = torch.zeros_like(f)
        pkg.msmg_solve(S.ctx, f, x64, RTOL, 3000, 0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, info64 = pkg.msmg_solve(S.ctx, f, x64, RTOL, 3000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        rec["fp64"] = {"iterations": info64[0]["iterations"], "ms_per_step": a.elapsed_time(b),
                       "true_rel_residual": info64[0]["true_rel_residual"]}
        S.close()
        return rec, lam

    recs = {}
    recs["strategy1_Lcc12"], _ = measure(dict(n_eig=[12, 12]))
    recs["strategy1_Lcc24"], (lam1, lam2) = measure(dict(n_eig=[12, 24]), export=True)
    lam1, lam2 = lam1.ravel(), lam2.ravel()
    lam2 = lam2[np.isfinite(lam2)]
    for name, k1, k2 in (("strategy2_Bcc_mean12", 12, 12), ("strategy2_Bcc_mean8", 12, 8),
                         ("strategy2_Bc_mean8_Bcc_mean12", 8, 12)):
        B1 = float(np.quantile(lam1, k1 / 12.0)) if k1 < 12 else 0.0
        B2 = float(np.quantile(lam2, k2 / 24.0))
        recs[name], _ = measure(dict(n_eig=[12, 24], eig_threshold=[B1, B2]))
        recs[name]["B"] = [B1, B2]
    best = "strategy2_Bcc_mean12"
    line = {"metric": METRIC, "value": recs[best]["value"], "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": recs[best]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": STRAT2_WORKLOAD, "form": "mixed",
                                             "l2": "flushed before each step (256 MiB write); working set > L2"},
            "runs": recs}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


NET_WORKLOAD = ("warm-start network forward pass (the a16 products): 8192 level-1 elements of 8^3 cells, "
                "512 -> 1024 -> 1024 -> 5 x 512 with ReLU, BF16 operands, FP32 accumulation; tensor cores "
                "(tcgen05, widths multiples of 64) against the CUDA-core products (hidden widths 1000)")


def run_network(args, world, rank, local):
    """Forward throughput of the warm-start network: the tcgen05 products against
    the CUDA-core products of a network of nearly the same size."""
    import torch
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    B = 8192
    stream = torch.cuda.current_stream()
    x = torch.randn(B, 512, device="cuda", dtype=torch.float32) * 0.5
    out = {}
    for name, hidden in (("tensor_cores", (1024, 1024)), ("cuda_cores", (1000, 1000))):
        net = pkg.WarmStartNet(n_in=512, hidden=hidden, n_vec=5, batch_max=B, seed=1)
        for _ in range(max(1, args.warmup)):
            net.forward(x)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            net.forward(x)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        flops = 2.0 * B * (512 * hidden[0] + hidden[0] * hidden[1] + hidden[1] * 5 * 512)
        out[name] = {"ms_per_forward": ms, "tflops": flops / (ms * 1e-3) / 1e12, "hidden": list(hidden)}
        if name == "tensor_cores":
            # each product alone, CUDA events on its own launch, L2 flushed before each pass
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
            dims = (512, hidden[0], hidden[1], 5 * 512)
            acc = [0.0, 0.0, 0.0]
            for k in range(args.steps):
                flush.fill_(float(k))
                t = pkg.msmg_net_time_products(net.handle, x, stream)
                acc = [u + v for u, v in zip(acc, t)]
            per = []
            for l in range(3):
                ms_l = acc[l] / args.steps
                fl = 2.0 * B * dims[l] * dims[l + 1]
                per.append({"M": B, "N": dims[l + 1], "K": dims[l], "ms": ms_l, "tflops": fl / (ms_l * 1e-3) / 1e12})
            out[name]["products"] = per
        net.close()
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        peak = 1900.0
    tc = out["tensor_cores"]
    line = {"metric": "warm-start network forward TFLOP/s (BF16 operands, FP32 accumulation)", "value": tc["tflops"],
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tc["ms_per_forward"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic", "config": {"workload": NET_WORKLOAD, "batch": B},
            "roofline": {"bound": "tensor", "kernel": "k_gemm_tc (layer 3, the largest product)",
                         "achieved": tc["products"][2]["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": tc["products"][2]["tflops"] / peak, "peak_source": "measured cuBLAS bf16 burst",
                         "traffic": None},
            "forms": out, "speedup_over_cuda_cores": out["cuda_cores"]["ms_per_forward"] / tc["ms_per_forward"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


IMPES_WORKLOAD = ("two-phase IMPES (Section 6) on the SPE10 grid shape: 60 x 220 x 85 cells of 20 x 10 x 2 ft, "
                  "85 layers of 60 x 220 lognormal lattices with sinuous channels (the layered recipe, seed 100), "
                  "kappa_z = kappa_x / 10; porosity U(0.05, 0.3); producers at BHP 4000 in the four corner columns "
                  "(well index of Section 6, r_w = 1 ft), an injector in the centre column; mu_w 0.3, mu_o 3.0, "
                  "s_wc = s_or = 0.2; DS_max 0.001, M = 50 sub-steps; 4x4x5 elements, ratio (3, 5, 1), 3 levels, "
                  "4 eigenvectors per local problem, mixed form, rtol 1e-9, pressure warm-started")


def run_impes(args, world, rank, local):
    """Pressure steps of the improved IMPES scheme: mobility terms, set-up, warm-started
    solve, velocity and M saturation sub-steps per step, all in the library's kernels."""
    import torch
    import fields
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    from math import log, pi, sqrt
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nz, ny, nx = 85, 220, 60
    shape = (nz, ny, nx)
    h = (20.0, 10.0, 2.0)
    kx = fields.layered_channels(shape, seed=100)
    kappa = torch.tensor(np.stack([kx, kx, 0.1 * kx]), device=dev)
    rng = np.random.default_rng(100)
    phi = torch.tensor(rng.uniform(0.05, 0.3, size=shape), device=dev)
    r1 = sqrt(9 * h[0] ** 2 + h[1] ** 2) / 2
    r2 = sqrt(h[0] ** 2 + 9 * h[1] ** 2) / 2
    wi_val = (1 / h[0] ** 2 + 1 / h[1] ** 2) / ((2 / pi) * (h[1] / h[0] * log(r1) + h[0] / h[1] * log(r2)) - 1)
    wi = torch.zeros(shape, dtype=torch.float64, device=dev)
    for (j, i) in ((0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1)):
        wi[:, j, i] = wi_val
    q = torch.zeros(shape, dtype=torch.float64, device=dev)
    q[:, ny // 2, nx // 2] = 1.0e3
    S = torch.full(shape, 0.2, dtype=torch.float64, device=dev)
    fl = pkg.make_fluid()
    p = None
    steps = []
    n = nx * ny * nz
    ev = lambda: torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    n_steps = max(args.steps, 1) + max(args.warmup, 0)
    sol = None
    for k in range(n_steps):
        e = [ev() for _ in range(5)]
        e[0].record(stream)
        ke, w, b = pkg.msmg_impes_pressure_terms(fl, S, kappa, wi, q, 4000.0)
        e[1].record(stream)
        if sol is None:
            sol = pkg.Solver(ke, pkg.Options(n_levels=3, block=(4, 4, 5), ratio=[(3, 5, 1)], n_eig=[4, 4],
                                             precision=pkg.MIXED, eig_tol=1e-8, cell_diag=w), h=h)
        else:                                   # the operator changed: set up again in place
            sol.refresh(ke, cell_diag=w)
        e[2].record(stream)
        p, info, _ = sol.solve(b, rtol=1e-9, x0=p)
        e[3].record(stream)
        v, bal = sol.velocity(p, b)
        dt = pkg.msmg_impes_transport(sol.ctx, fl, v, p, w, 4000.0, q, phi, S, 50, 1e-3)
        e[4].record(stream)
        torch.cuda.synchronize()
        i0 = sol.info
        steps.append({"iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
                      "terms_ms": e[0].elapsed_time(e[1]), "setup_ms": e[1].elapsed_time(e[2]),
                      "setup_ms_library": i0["setup_ms"], "eig_ms": i0["eig_ms"],
                      "solve_ms": e[2].elapsed_time(e[3]), "velocity_transport_ms": e[3].elapsed_time(e[4]),
                      "dt": dt, "S_max": float(S.max()), "balance": bal[0] / max(bal[1], 1e-300)})
    sol.close()
    timed = steps[max(args.warmup, 0):]
    solve_ms = float(np.mean([s_["solve_ms"] for s_ in timed]))
    step_ms = float(np.mean([s_["terms_ms"] + s_["setup_ms"] + s_["solve_ms"] + s_["velocity_transport_ms"]
                             for s_ in timed]))
    line = {"metric": "IMPES pressure-solve DOF/s (rtol 1e-9, warm start) and time per IMPES step", "value": n / (solve_ms * 1e-3),
            "unit": "DOF/s", "n_gpus": world, "steps": len(timed), "warmup": max(args.warmup, 0),
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic", "config": {"workload": IMPES_WORKLOAD},
            "steps_record": steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


SCALE_N = 1024
SCALE_WORKLOAD = ("1024^3 lognormal field (exponential covariance, correlation length 0.1, 1024 random Fourier "
                  "modes in FP32 on the GPU, seed 5) rescaled to contrast 1e6; corner source/sink; 8^3 elements, "
                  "7 levels (ratio 2), 4 eigenvectors per local problem; PCG rtol 1e-8")


def run_scale(args, world, rank, local):
    """The single-GPU limit: a 1024^3 problem in the mixed form."""
    import torch
    import fields
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    pkg.load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = SCALE_N
    n = N ** 3
    # stated: 5 levels as specified (coarsest 16^3 elements x 4 = 16384 unknowns, a 2 GiB dense
    # pseudo-inverse); tuned: 7 levels (coarsest 256 unknowns)
    nl = 5 if args.hierarchy == "stated" else 7
    opts = pkg.Options(n_levels=nl, block=(8, 8, 8), ratio=[(2, 2, 2)] * (nl - 2), n_eig=[4] * (nl - 1),
                       precision=pkg.MIXED, eig_tol=1e-8, autotune=True)
    need = pkg.msmg_workspace_size(pkg.make_grid((N, N, N)), opts.to_c(), 1)
    free, total = torch.cuda.mem_get_info()
    vec_bytes = 2 * 8 * n + 4 * n                       # rhs, x (FP64) and kappa (FP32)
    if need + vec_bytes + (8 << 30) > free:
        print(json.dumps({"workload": SCALE_WORKLOAD, "skipped": f"needs {(need + vec_bytes) / 2**30:.1f} GiB, "
                          f"{free / 2**30:.1f} GiB free"}), flush=True)
        return 0
    t0 = time.perf_counter()
    kappa = fields.grf_lognormal_device((N, N, N), seed=5, contrast=1e6, device="cuda")
    torch.cuda.synchronize()
    t_field = time.perf_counter() - t0
    S = pkg.Solver(kappa, opts)
    info0 = S.info
    del kappa
    f = torch.tensor(rhs((N, N, N)), device=dev)
    x = torch.zeros_like(f)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pkg.msmg_solve(S.ctx, f, x, RTOL, 2000, 0)
    torch.cuda.synchronize()
    ms, info = [], None
    for k in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, info = pkg.msmg_solve(S.ctx, f, x, RTOL, 2000, 0)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    step = max_over_ranks(world, float(np.mean(ms)))
    kt = S.time_kernels(reps=3)
    line = {"metric": METRIC, "value": world * n / (step * 1e-3), "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": SCALE_WORKLOAD.replace("7 levels", f"{nl} levels"), "hierarchy": args.hierarchy,
                       "form": "mixed", "l2": "working set far above L2"},
            "iterations": info[0]["iterations"], "true_rel_residual": info[0]["true_rel_residual"],
            "converged": info[0]["converged"], "setup_ms": info0["setup_ms"], "eig_ms": info0["eig_ms"],
            "eig_iterations_max": info0["eig_iterations_max"], "workspace_gib": need / 2**30,
            "field_s": t_field, "kernel_ms": kt, "gpu_launches": int(info[0]["kernel_launches"])}
    S.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_profile(args):
    """Short run for ncu: set-up of the default workload, then one solve capped at
    ``--max-iter`` PCG iterations in the chosen form."""
    import torch
    import paper_2403_19342_gb300 as pkg
    from paper_2403_19342_gb300 import build as _build
    _build.build()
    kappa = torch.tensor(field(), device="cuda")
    f = torch.tensor(rhs(kappa.shape), device="cuda")
    x = torch.zeros_like(f)
    prec = pkg.MIXED if args.form == "mixed" else pkg.FP64
    S = pkg.Solver(kappa, pkg.Options(n_levels=N_LEVELS, block=BLOCK, ratio=RATIO, n_eig=N_EIG, precision=prec,
                                      eig_tol=1e-8, autotune=True),
                   n_rhs=BATCH_RHS if args.form == "mixed" else 1, tuning_cache=args.tuning_cache)
    st, info = pkg.msmg_solve(S.ctx, f, x, RTOL, args.max_iter, 0)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.form, "iterations": info[0]["iterations"],
                      "kernel_launches": info[0]["kernel_launches"]}))
    S.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="short run for ncu (no timing output)")
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--max-iter", type=int, default=4)
    ap.add_argument("--workload", default="inclusions",
                    choices=["inclusions", "batched", "layered", "scale", "strategy2", "network", "impes"])
    ap.add_argument("--hierarchy", default="tuned", choices=["tuned", "stated"],
                    help="layered / scale: the tuned hierarchy or the one the configuration states")
    ap.add_argument("--tuning-cache", default=os.path.join(os.environ.get("TMPDIR", "/tmp"), "msmg_tuning.json"),
                    help="autotune cache (JSON): a later run, e.g. under a profiler, reuses the variants found")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    world, rank, local = dist_setup() if args.impl == "gpu" else (int(os.environ.get("WORLD_SIZE", "1")),
                                                                   int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    run = {"batched": run_batched, "layered": run_layered, "scale": run_scale,
           "strategy2": run_strategy2, "network": run_network, "impes": run_impes}.get(args.workload, run_gpu)
    rc = run(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
