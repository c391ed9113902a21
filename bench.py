#!/usr/bin/env python
"""Benchmark of the GB300 modal DG solver (arXiv:1602.09079).

Workload (one "step" = one SSP-RK3 step of the whole hot path): driven
subsonic turbulence on a periodic 128^3 box, order 3 (degree 2, 10 modes
per variable), gamma = 5/3, warm start rho = 1, p = 1/gamma with a
solenoidal velocity field at rms Mach 0.3 on the driving modes (seed 1234),
OU-driven solenoidal forcing on 1 <= |n| <= 2 (seed 1234), CFL 0.3. Each
step: CFL reduction (dg_cfl_dt), three fused stages (face fluxes, volume
quadrature + projection + stage combination + positivity limiter), and the
isothermal energy reset (dg_energy_reset).

Metric: DOF-updates per second per RK stage = cells x N(k) x 3 stages x
steps / time. The headline value is the FP32-mixed path (FP64 state, RK
accumulation, limiter and reductions); the plain FP64 path is reported
beside it with the mixed path's L2 error against it.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of cells of the same workload (the oracle is the baseline here).
Multi-GPU (torchrun): independent replicas, one per rank; value = all
ranks' DOF-updates / max time over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

GAMMA = 5.0 / 3.0
MACH = 0.3
SEED = 1234


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=128, help="cells per axis")
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--courant", type=float, default=0.3)
    ap.add_argument("--flux", choices=["hllc", "exact"], default="hllc",
                    help="numerical flux: HLLC or the exact Riemann solver")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--err-steps", type=int, default=None,
                    help="steps of the untimed mixed-vs-FP64 error run at a fixed dt (default: the "
                         "configurations' lengths, 200 at order 3 and 100 at order 4)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="convergence sweep of the smooth diagonal density wave (16^3..64^3, orders 2..4, t = 1)")
    ap.add_argument("--sweep-max-cells", type=int, default=64 ** 3 * 10 // 4,
                    help="skip (n, order) pairs with n^3 N(k) above this many DOF per variable x 4")
    ap.add_argument("--indicator", action="store_true",
                    help="learned troubled-cell indicator at size: train on the GPU (32^3 label runs), then "
                         "recall, misses and gated vs ungated step time on held-out 128^3 supersonic "
                         "turbulence and a Sod tube (config 5)")
    ap.add_argument("--ind-train-n", type=int, default=32)
    ap.add_argument("--ind-train-steps", type=int, default=3000)
    ap.add_argument("--ind-timed-steps", type=int, default=10)
    ap.add_argument("--ind-network", action="store_true",
                    help="only time the indicator network's forward and backward kernels on 1M random rows")
    ap.add_argument("--precisions", default="fp64,mixed",
                    help="comma list of fp64,mixed (the first listed of mixed/fp64 is the headline)")
    return ap.parse_args()


def workload_config(args, precision):
    n = args.n
    N = (args.order) * (args.order + 1) * (args.order + 2) // 6
    return {
        "workload": (f"driven subsonic turbulence, periodic {n}^3 box, order {args.order} "
                     f"(degree {args.order - 1}), gamma 5/3, warm start rms Mach {MACH} "
                     f"(seed {SEED}), OU solenoidal forcing on 1<=|n|<=2, energy reset every "
                     f"step, CFL {args.courant}"
                     + (", exact Riemann solver flux" if getattr(args, "flux", "hllc") == "exact" else "")),
        "flux": getattr(args, "flux", "hllc"),
        "cells": n ** 3,
        "dof_per_cell_per_var": N,
        "precision": precision,
        "l2": (f"state {5 * N * 8 * n ** 3 / 1e6:.0f} MB per buffer, "
               + ("larger than the 129 MB L2 (no flush needed)" if 5 * N * 8 * n ** 3 > 129e6
                  else "smaller than the 129 MB L2 (not a timing configuration)")),
    }


# ------------------------------------------------------------ distributed
def dist_init(use_cuda):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

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
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ setup
def build_state_host(args):
    """Canonical initial state from the oracle's projection (reference arm)."""
    import oracle
    n = (args.n,) * 3
    o = oracle.Oracle(n, args.order - 1, GAMMA)
    fn = syn.solenoidal_velocity(seed=SEED, mach=MACH, gamma=GAMMA)
    return o, o.project_fn(fn)


def driving(args):
    from paper_1602_09079_gb300.forcing import OUDriving
    nv = syn.driving_modes(1.0, 2.0)
    cs = math.sqrt(GAMMA * (1.0 / GAMMA) / 1.0)
    t_s = 1.0 / (2.0 * MACH * cs)  # half the eddy turnover time, L = 1 (Sect. 3.1)
    z = syn.ou_noise(SEED, 2, len(nv))
    # amplitude: rms acceleration ~ (M c)^2 k_drive, the order that sustains
    # rms Mach M against dissipation at the driving scale (fixed here; the
    # paper rescales it to the target Mach number)
    amp = (MACH * cs) ** 2 * 2 * math.pi * 1.5
    drv = OUDriving(nv, t_s, 0.1 * t_s, amp, z[0])
    drv.update(z[1])
    return drv


def roofline_entry(kind, achieved, peak, unit, bound, traffic=None):
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if peak else None, "traffic": traffic}


def step_roofline(k, mixed, nc, ms_per_step, hbm_gbs):
    """Whole-step roofline: the algorithmic work of the step's three RK
    stages (roofline.step_min_bytes: read y_s, y_0, write y_{s+1} in FP64;
    3 x roofline.stage_flops, sum-factorised) plus the energy reset (read the
    density and momentum modes and the energy mean, write the energy modes)
    and the CFL reduction (five means), over the measured step time; bound
    by the larger of the ALU time (FP32 peak on the mixed path, FP64 on the
    plain one) and the HBM time."""
    from paper_1602_09079_gb300 import roofline as rl
    N = (k + 1) * (k + 2) * (k + 3) // 6
    sec = ms_per_step * 1e-3
    byts = (rl.step_min_bytes(k) + (4 * N + 1 + N) * 8 + 5 * 8) * nc
    flops = 3 * rl.stage_flops(k, True) * nc
    peak = rl.FP32_PEAK if mixed else rl.FP64_PEAK
    t_alu = flops / peak
    t_hbm = byts / (hbm_gbs * 1e9) if hbm_gbs else None
    out = {"bytes_per_step": byts, "flops_per_step": flops, "achieved_gbs": byts / sec / 1e9,
           "achieved_tflops": flops / sec / 1e12, "peak_source": rl.PEAK_SOURCE,
           "impl_bytes_per_step": rl.step_bytes(k, mixed) * nc}
    if t_hbm is None:
        out.update({"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None})
    elif t_alu >= t_hbm:
        out.update({"bound": "alu", "achieved": flops / sec / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": t_alu / sec})
    else:
        out.update({"bound": "hbm", "achieved": byts / sec / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": t_hbm / sec})
    return out


def ncu_traffic():
    """DRAM bytes per cell per launch of the profiled kernels, from the ncu
    capture summarised in profiles/ncu_traffic.json (a smaller mesh of the
    same workload; traffic scales with the cells processed)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            return json.load(f).get("kernels", {})
    except (OSError, ValueError):
        return {}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


# --------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_1602_09079_gb300 as dgm
    from paper_1602_09079_gb300 import roofline as rl

    world, rank, local = dist_init(True)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dgm.load()
    n = (args.n,) * 3
    k = args.order - 1
    s = dgm.Solver(n, args.order, GAMMA, forcing=True)
    s.set_flux(dgm.DG_FLUX_EXACT if args.flux == "exact" else dgm.DG_FLUX_HLLC)
    N, nc = s.N, s.ncells
    fn = syn.solenoidal_velocity(seed=SEED, mach=MACH, gamma=GAMMA)
    s.project_fn(fn)
    drv = driving(args)
    s.set_forcing(drv.nvec, drv.ahat())
    w0_dev = torch.from_numpy(s.get_state()).to(dev)
    c_iso = math.sqrt(1.0 / GAMMA)  # p0/rho0 at the start state

    def one_step():
        dt = s.cfl_dt(args.courant)
        s.step(dt)
        s.energy_reset(c_iso, 1.0)

    results = {}
    precs = [p for p in ("fp64", "mixed") if p in args.precisions.split(",")]
    for prec_name in precs:
        prec = dgm.DG_PREC_FP64 if prec_name == "fp64" else dgm.DG_PREC_MIXED
        s.set_precision(prec)
        s.set_state(w0_dev)
        for _ in range(args.warmup):
            one_step()
        s.check()
        s.kernel_stats()  # reset counters
        clocks = Clocks(local)
        barrier(world)
        torch.cuda.synchronize()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        for _ in range(args.steps):
            one_step()
        e1.record(s.stream)
        torch.cuda.synchronize()
        barrier(world)
        ck = clocks.stop()
        s.check()
        stats = s.kernel_stats()
        ms = e0.elapsed_time(e1)
        ms_max = max_over_ranks(world, ms, dev)
        dof = float(nc) * N * 3 * args.steps
        dof_all = sum_over_ranks(world, dof, dev)
        # per-kernel timing pass (events around every launch, separate steps)
        s.set_timing(True)
        for _ in range(2):
            one_step()
        kst = s.kernel_stats()
        s.set_timing(False)
        results[prec_name] = {"ms": ms, "ms_max": ms_max, "dof_all": dof_all, "clocks": ck,
                              "launches": stats, "ktimes": kst}

    # mixed vs FP64 error at matched steps with a fixed dt
    s.set_precision(dgm.DG_PREC_FP64)
    s.set_state(w0_dev)
    dt_fix = s.cfl_dt(args.courant)
    err_steps = args.err_steps

    def fixed_run(prec):
        s.set_precision(prec)
        s.set_state(w0_dev)
        for _ in range(err_steps):
            s.step(dt_fix)
            s.energy_reset(c_iso, 1.0)
        s.check()
        return s.y.view(5, N, nc).clone()

    l2 = mx = None
    if err_steps > 0:
        y64 = fixed_run(dgm.DG_PREC_FP64)
        ymx = fixed_run(dgm.DG_PREC_MIXED)
        d = ymx - y64
        l2 = (torch.sqrt((d * d).sum(dim=(1, 2))) / torch.sqrt((y64 * y64).sum(dim=(1, 2)))).tolist()
        mx = (d.abs().amax(dim=(1, 2)) / y64.abs().amax(dim=(1, 2))).tolist()
        del y64, ymx, d

    # end-to-end through the public API with host buffers
    s.set_precision(dgm.DG_PREC_MIXED if "mixed" in results else dgm.DG_PREC_FP64)
    e2e_s = 0.0
    if args.e2e_steps > 0:
        host_in = torch.from_numpy(w0_dev.cpu().numpy()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            dgm.dg_set_state(s.ctx, host_in.data_ptr(), 0)
            one_step()
            dgm.dg_get_state(s.ctx, host_out.data_ptr(), 0)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        del host_in, host_out
    e2e_s = max(max_over_ranks(world, e2e_s, dev), 1e-30)
    e2e_dof = sum_over_ranks(world, float(nc) * N * 3 * args.e2e_steps, dev)
    state_bytes = 5 * N * nc * 8

    # roofline of the dominant kernel (volume) from the live per-launch timing
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    fp64_probe = dgm.dg_probe_fma_peak(True)
    fp32_probe = dgm.dg_probe_fma_peak(False)

    def kernel_roofline(prec_name, tsize):
        """Roofline of one RK stage: the stage kernels' time per stage (the
        fused kernel on the mixed path at degrees 2-3; face and volume kernels
        otherwise) against the method's algorithmic bytes (read y_s and y_0,
        write y_{s+1} in FP64) and sum-factorised flops of a stage
        (roofline.stage_roofline); traffic = the ncu DRAM bytes of the timed
        kernel per launch, with its ratio to the algorithmic bytes."""
        kst = results[prec_name]["ktimes"]
        nvol, msvol = kst["volume"]
        nface, msface = kst["face_flux"]
        stage_ms = (msvol + msface) / nvol
        peak = rl.FP32_PEAK if tsize == 4 else rl.FP64_PEAK
        e = rl.stage_roofline(k, True, nc, stage_ms, hbm, peak)
        e["peak_source"] = rl.PEAK_SOURCE
        fused = tsize == 4 and nface == 0
        if fused:
            kname = f"fused_f32_kernel<{k}, true, {1 if args.flux == 'exact' else 0}>"
            e["kernel"] = kname + " (stage, forcing; face fluxes, volume integral and stage update in one launch)"
            e["impl_bytes_per_launch"] = rl.fused_impl_bytes(k, True) * nc
        else:
            sumfact = k >= 2
            kname = (f"volume_f32_kernel<{k}, 1, 1>" if (tsize == 4 and k <= 2)
                     else f"volume_{('sfb_' if tsize == 4 else 'sf_') if sumfact else ''}kernel<{k}, "
                     f"{'double' if tsize == 8 else 'float'}, 1, 1>")
            e["kernel"] = kname + " (stage, forcing) + its face kernel"
            e["impl_bytes_per_launch"] = (rl.volume_bytes(k, tsize, True, shadow=tsize == 4)
                                          + rl.face_bytes(k, tsize)) * nc
        # the captured FP64 traffic is that of the HLLC face kernel: no entry
        # for the exact-flux path
        tr = None if (args.flux == "exact" and not fused) else ncu_traffic().get(kname)
        e["traffic"] = None
        if tr and not tr.get("stale"):
            e["traffic"] = tr["dram_bytes_per_cell"] * nc
            e["traffic_source"] = tr.get("source")
            e["traffic_over_algorithmic_bytes"] = e["traffic"] / e["bytes_per_launch"]
        tot = sum(v[1] for v in kst.values())
        e["share_of_step"] = {kk: (v[1] / tot if tot else None) for kk, v in kst.items()}
        e["ms_per_launch_by_class"] = {kk: (v[1] / v[0] if v[0] else None) for kk, v in kst.items()}
        return e

    head = "mixed" if "mixed" in results else "fp64"
    r_mx = results[head]
    r_64 = results.get("fp64", r_mx)
    value = r_mx["dof_all"] / (r_mx["ms_max"] * 1e-3)
    value64 = r_64["dof_all"] / (r_64["ms_max"] * 1e-3)
    launches = sum(v[0] for v in r_mx["launches"].values())

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(args, s.get_state(), drv, budget=args.cpu_seconds)

    if rank == 0:
        out = {
            "metric": "DG DOF-updates/sec per RK stage (FP32-mixed, FP64 RK accumulation; FP64 plain beside it)",
            "value": value,
            "unit": "DOF-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": r_mx["ms_max"] / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 (f64 state and accumulation)" if head == "mixed" else "f64",
            "data": "synthetic",
            "config": workload_config(args, head),
            "roofline": kernel_roofline(head, 4 if head == "mixed" else 8),
            "step_roofline": step_roofline(k, head == "mixed", nc, r_mx["ms_max"] / args.steps, hbm),
            "value_x5_variables": 5 * value,
            "fp64": {
                "value": value64,
                "unit": "DOF-updates/s",
                "ms_per_step": r_64["ms_max"] / args.steps,
                "dtype": "f64",
                "roofline": kernel_roofline("fp64", 8) if "fp64" in results else None,
                "step_roofline": (step_roofline(k, False, nc, r_64["ms_max"] / args.steps, hbm)
                                  if "fp64" in results else None),
                "clocks": r_64["clocks"],
                "gpu_launches": sum(v[0] for v in r_64["launches"].values()),
            },
            "speedup_mixed_over_fp64": value / value64,
            "mixed_vs_fp64_error": {"steps": err_steps, "dt": dt_fix,
                                    "l2_rel_per_var": l2, "max_coef_rel_per_var": mx},
            "e2e": {"value": (e2e_dof / e2e_s) if args.e2e_steps > 0 else None, "unit": "DOF-updates/s",
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                    "note": "dg_set_state from pinned host + step + dg_get_state to pinned host, per step"},
            "gpu_launches": launches,
            "launches_by_class": {kk: v[0] for kk, v in r_mx["launches"].items()},
            "clocks": r_mx["clocks"],
            "probe_fma_tflops": {"fp64": fp64_probe / 1e12, "fp32": fp32_probe / 1e12},
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    barrier(world)


# ----------------------------------------------------------- CPU oracle
def cpu_baseline(args, w_canon, drv, budget=12.0, sample=4096):
    """The FP64 oracle on the host cores: R (all five variables) and the
    limiter at a fixed random sample of cells of the same state, i.e. one RK
    stage's work on the sample."""
    import oracle
    o = oracle.Oracle((args.n,) * 3, args.order - 1, GAMMA)
    o.set_forcing(drv.nvec, drv.ahat())
    cells = syn.sample_cells(o.ncells, sample, seed=3)
    N = o.N
    t0 = time.perf_counter()
    reps = 0
    while True:
        o.rhs_cells(w_canon, cells)
        o.limit_cells(w_canon, cells)
        reps += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = (time.perf_counter() - t0) / reps
    return {"value": len(cells) * N / dt, "unit": "DOF-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"R + limiter on {len(cells)} random cells of the {args.n}^3 state, {reps} reps"}


def run_reference(args):
    world, rank, local = dist_init(False)
    if rank != 0:
        return
    import oracle
    oracle.build()
    o, w = build_state_host(args)
    drv = driving(args)
    o.set_forcing(drv.nvec, drv.ahat())
    cells = syn.sample_cells(o.ncells, 8192, seed=3)
    for _ in range(args.warmup):
        o.rhs_cells(w, cells)
        o.limit_cells(w, cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.rhs_cells(w, cells)
        o.limit_cells(w, cells)
    el = time.perf_counter() - t0
    value = len(cells) * o.N * args.steps / el
    sample = f"R + limiter on {len(cells)} random cells of the {args.n}^3 state per step"
    print(json.dumps({
        "impl": "reference",
        "metric": "DG DOF-updates/sec per RK stage (FP32-mixed, FP64 RK accumulation; FP64 plain beside it)",
        "value": value, "unit": "DOF-updates/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, "fp64 (CPU oracle)"),
        "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------- learned indicator (config 5)
def _ind_snapshots(dgm, torch, fn, n, steps, every, courant=0.15, precision=0):
    """Runs of the solver with the plain limiter from the state fn; every
    `every` steps the features and plain-indicator labels of the cells that
    fail the limiter's screen (dg_indicator_capture)."""
    order = 3
    nf, F, npar, work = dgm.dg_indicator_sizes(order)
    s = dgm.Solver((n, n, n), order, GAMMA)
    s.set_precision(precision)
    s.project_fn(fn)
    X = torch.empty((s.ncells, F), dtype=torch.bfloat16, device="cuda")
    fl = torch.empty(s.ncells, dtype=torch.int8, device="cuda")
    sc = torch.empty(s.ncells, dtype=torch.uint8, device="cuda")
    xs, ys = [], []
    for it in range(steps):
        dt = s.cfl_dt(courant)
        s.step(dt)
        if it % every == every - 1:
            dgm.dg_indicator_capture(s.ctx, dt, X, fl, sc)
            m = sc.bool()
            if int(((fl != 0) & ~m).sum()) != 0:
                raise RuntimeError("the limiter screen missed a troubled cell")
            xs.append(X[m].clone())
            ys.append((fl[m] != 0).float())
    s.check()
    del s, X, fl, sc
    torch.cuda.empty_cache()
    return torch.cat(xs), torch.cat(ys)


def _ind_init(F, seed):
    """He-uniform weights, zero biases; flat layout [W1 b1 W2 b2 w3 b3]."""
    H = 64
    rng = np.random.default_rng(seed)
    lim1, lim2 = math.sqrt(6.0 / F), math.sqrt(6.0 / H)
    parts = [rng.uniform(-lim1, lim1, H * F), np.zeros(H), rng.uniform(-lim2, lim2, H * H), np.zeros(H),
             rng.uniform(-lim2, lim2, H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def _ind_network(dgm, torch, order, rows=1 << 20, reps=10):
    """Forward and backward kernels of the indicator network on `rows` random
    BF16 feature rows (CUDA events, mean of `reps` launches after 3 warm-up
    launches of each), with their rooflines: algorithmic HBM bytes (the
    feature rows read once, the logits or labels) and tensor flops per row
    (forward F*H + H*H + H MACs; backward the forward again plus dW2, dH1,
    dW1 and the output layer's gradients), against the measured HBM copy and
    cuBLAS bf16 peaks."""
    H = 64
    nf, F, npar, work = dgm.dg_indicator_sizes(order)
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    X = torch.randn(rows, F, device="cuda", generator=g).to(torch.bfloat16)
    y = (torch.rand(rows, device="cuda", generator=g) < 0.1).float()
    P = torch.from_numpy(_ind_init(F, 3)).cuda()
    G = torch.zeros(npar + 1, dtype=torch.float32, device="cuda")
    Wk = torch.empty(work, dtype=torch.uint8, device="cuda")
    logits = torch.empty(rows, dtype=torch.float32, device="cuda")
    for _ in range(3):
        dgm.dg_indicator_forward(order, X, rows, P, logits, 0)
        dgm.dg_indicator_backward(order, X, y, rows, 1.0, P, G, Wk, work, 0)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(reps):
        dgm.dg_indicator_forward(order, X, rows, P, logits, 0)
    ev[1].record()
    for _ in range(reps):
        dgm.dg_indicator_backward(order, X, y, rows, 1.0, P, G, Wk, work, 0)
    ev[2].record()
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
    pk = measured_peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    tc = pk.get("bf16_tflops", 1900.0)
    fwd_mac = F * H + H * H + H
    bwd_mac = fwd_mac + H * H + H * H + F * H + 2 * H
    out = {"rows": rows, "features": F, "hidden": H, "kernel": "mma.sync m16n8k16 bf16, fp32 accumulate"}
    for name, ms, mac in (("forward", fwd_ms, fwd_mac), ("backward", bwd_ms, bwd_mac)):
        byts = rows * (2 * F + 4)
        flops = rows * 2 * mac
        t_hbm, t_tc = byts / (hbm * 1e9), flops / (tc * 1e12)
        out[name] = {"ms": ms, "bytes": byts, "flops": flops, "gbs": byts / (ms * 1e6),
                     "tflops": flops / (ms * 1e9), "bound": "hbm" if t_hbm >= t_tc else "tensor",
                     "frac": max(t_hbm, t_tc) / (ms * 1e-3),
                     "peaks": f"HBM {hbm} GB/s, bf16 {tc} TFLOP/s (measured)"}
    return out


def run_indicator(args):
    """Config 5: the BF16 troubled-cell network trained on the GPU by the
    library's backward and Adam kernels from plain-indicator labels of 32^3
    supersonic-turbulence and Sod-tube runs (FP64 path), its threshold set so
    that 99% of the validation runs' troubled cells pass; then at 128^3, on
    held-out supersonic turbulence (rms Mach 2.5) and a held-out Sod tube:
    recall and misses judged by the plain indicator, and the mixed-path step
    time (CUDA events on the solver's stream, the gate's features and network
    included) with the network gating the full limiter vs without it."""
    import torch
    import paper_1602_09079_gb300 as dgm
    dgm.load()
    order, n_tr, n = 3, args.ind_train_n, args.n
    nf, F, npar, work = dgm.dg_indicator_sizes(order)
    t0 = time.perf_counter()

    def data(specs, nn):
        xs, ys = [], []
        for kind, seed, mach in specs:
            if kind == "super":
                x, y = _ind_snapshots(dgm, torch, syn.supersonic_velocity(seed, mach, GAMMA), nn, 240, 30)
            else:
                x, y = _ind_snapshots(dgm, torch, syn.sod_tube(seed, GAMMA)[0], nn, 120, 20)
            xs.append(x)
            ys.append(y)
        return torch.cat(xs), torch.cat(ys)

    Xtr, ytr = data([("super", 1, 2.0), ("super", 2, 2.5), ("super", 3, 3.0), ("super", 4, 2.5),
                     ("sod", 1, 0), ("sod", 2, 0)], n_tr)
    Xva, yva = data([("super", 9, 2.5), ("sod", 6, 0)], n_tr)
    P = torch.from_numpy(_ind_init(F, 70)).cuda()
    m1, m2 = torch.zeros_like(P), torch.zeros_like(P)
    G = torch.zeros(npar + 1, dtype=torch.float32, device="cuda")
    Wk = torch.empty(work, dtype=torch.uint8, device="cuda")
    pos = float(ytr.sum())
    pw = max(1.0, (len(ytr) - pos) / max(pos, 1.0))
    losses = []
    torch.cuda.synchronize()
    tt = time.perf_counter()
    for step in range(1, args.ind_train_steps + 1):
        dgm.dg_indicator_backward(order, Xtr, ytr, len(ytr), pw, P, G, Wk, work, 0)
        if step in (1, args.ind_train_steps):
            losses.append(float(G[npar]))
        dgm.dg_indicator_adam(P, m1, m2, G, npar, 3e-3, 0.9, 0.999, 1e-8, step, 0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - tt

    def prob(X):
        out = torch.empty(len(X), dtype=torch.float32, device="cuda")
        dgm.dg_indicator_forward(order, X, len(X), P, out, 0)
        return torch.sigmoid(out)

    thr = float(torch.quantile(prob(Xva)[yva > 0].float(), 0.01))
    thr = max(min(thr, 0.999), 1e-12)
    rows_tr = len(ytr)
    del Xtr, ytr, Xva, yva
    torch.cuda.empty_cache()

    out = {"metric": "learned troubled-cell indicator at 128^3, order 3 (config 5)", "n": n, "order": order,
           "train": {"n": n_tr, "rows": rows_tr, "adam_steps": args.ind_train_steps, "loss_first_last": losses,
                     "seconds": train_s, "pos_weight": pw},
           "threshold": thr, "network": _ind_network(dgm, torch, order), "workloads": {}}
    for kind, seed, mach in (("supersonic turbulence, rms Mach 2.5 (seed 7)", 7, 2.5),
                             ("Sod tube (seed 5)", 5, 0.0)):
        fn = syn.supersonic_velocity(seed, mach, GAMMA) if mach > 0 else syn.sod_tube(seed, GAMMA)[0]
        # held-out recall and misses at 128^3: FP64 runs, captures every 20 steps
        Xte, yte = _ind_snapshots(dgm, torch, fn, n, 60, 20)
        pte = prob(Xte)
        sel = pte >= thr
        tro = yte > 0
        rec = {"captured_rows": len(yte), "troubled": int(tro.sum()),
               "recall": (float((sel & tro).sum()) / float(tro.sum())) if int(tro.sum()) > 0 else None,
               "misses": int((~sel & tro).sum()), "false_flags": int((sel & ~tro).sum()),
               "evaluated_fraction": float(sel.float().mean())}
        del Xte, yte, pte, sel, tro
        torch.cuda.empty_cache()
        # timing at 128^3 on the mixed path from the same evolved state
        s = dgm.Solver((n, n, n), order, GAMMA)
        s.set_precision(dgm.DG_PREC_MIXED)
        s.project_fn(fn)
        for _ in range(20):
            s.step(s.cfl_dt(0.15))
        s.check()
        w = s.get_state()
        dt = s.cfl_dt(0.15)
        timing = {}
        for gate in (False, True):
            s2 = dgm.Solver((n, n, n), order, GAMMA)
            s2.set_precision(dgm.DG_PREC_MIXED)
            s2.set_state(w)
            if gate:
                dgm.dg_set_indicator(s2.ctx, P, thr)
            for _ in range(args.warmup):
                s2.step(dt)
            s2.set_state(w)
            s2.limit()  # the step's input limited before the timed region, as after any step
            dgm.dg_limiter_counts(s2.ctx)  # reads and clears the totals
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s2.stream)
            for _ in range(args.ind_timed_steps):
                s2.step(dt)
            e1.record(s2.stream)
            torch.cuda.synchronize()
            ok = True
            try:
                s2.check()
            except dgm.DGError:
                ok = False
            q1 = dgm.dg_limiter_counts(s2.ctx)
            s2.set_timing(True)
            s2.set_state(w)
            s2.limit()
            s2.kernel_stats()
            for _ in range(2):
                s2.step(dt)
            kst = s2.kernel_stats()
            s2.set_timing(False)
            timing["gated" if gate else "ungated"] = {
                "ms_per_step": e0.elapsed_time(e1) / args.ind_timed_steps,
                "screen_failures_per_step": q1[0] / args.ind_timed_steps,
                "full_limiter_cells_per_step": q1[1] / args.ind_timed_steps,
                "limiter_ms_per_step": kst["limiter"][1] / 2, "stage_ms_per_step": kst["volume"][1] / 2,
                "positivity_ok": ok}
            del s2
            torch.cuda.empty_cache()
        timing["speedup_gated"] = timing["ungated"]["ms_per_step"] / timing["gated"]["ms_per_step"]
        out["workloads"][kind] = {"heldout_fp64_captures": rec, "mixed_step_timing": timing, "dt": dt}
        del s
        torch.cuda.empty_cache()
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out))


def l2_density_error(w, k, n, exact, nq=6):
    """L2 error of the density polynomial against exact(x, y, z) with an
    nq-point Gauss rule per axis per cell (numpy Legendre basis)."""
    import numpy.polynomial.legendre as npl
    modes = [(u, v, d - u - v) for d in range(k + 1) for u in range(d, -1, -1) for v in range(d - u, -1, -1)]
    xg, wg = npl.leggauss(nq)
    P = np.array([[math.sqrt(2 * u + 1) * npl.legval(x, [0] * u + [1]) for x in xg] for u in range(k + 1)])
    dx = 1.0 / n
    X = (np.arange(n)[:, None] + 0.5 + 0.5 * xg[None, :]) * dx
    W = (wg[:, None, None] * wg[None, :, None] * wg[None, None, :]) * (dx / 2) ** 3
    err = 0.0
    for iz in range(n):  # one z-slab at a time keeps memory small
        rho = np.zeros((n, n, nq, nq, nq))
        for l, (u, v, ww) in enumerate(modes):
            rho += w[iz, :, :, 0, l][..., None, None, None] * (
                P[u][None, None, None, None, :] * P[v][None, None, None, :, None] * P[ww][None, None, :, None, None])
        ex = exact(X[None, :, None, None, :], X[:, None, None, :, None], X[iz][None, None, :, None, None])
        err += np.sum((rho - ex) ** 2 * W[None, None])
    return math.sqrt(err)


def run_sweep(args):
    """Plain FP64 convergence sweep: rho = 1 + 0.2 sin(2 pi (x+y+z)), v = (1,1,1),
    p = 1, gamma = 5/3, SSP-RK3 at CFL 0.3 to t = 1, where the exact solution
    equals the initial profile."""
    import torch
    import paper_1602_09079_gb300 as dgm
    dgm.load()
    fn = syn.smooth_wave_diag(GAMMA)
    out = {"workload": "smooth diagonal density wave, FP64, t = 1", "runs": []}
    for order in (2, 3, 4):
        k = order - 1
        N = order * (order + 1) * (order + 2) // 6
        errs = []
        for n in (16, 32, 64):
            if n ** 3 * N > args.sweep_max_cells * 4:
                out["runs"].append({"n": n, "order": order, "skipped": "above --sweep-max-cells"})
                continue
            s = dgm.Solver((n, n, n), order, GAMMA)
            s.project_fn(fn)
            t, steps, t0 = 0.0, 0, time.perf_counter()
            while t < 1.0 - 1e-14:
                dt = min(s.cfl_dt(args.courant), 1.0 - t)
                s.step(dt)
                t += dt
                steps += 1
            s.check()
            wall = time.perf_counter() - t0
            err = l2_density_error(s.get_state(), k, n, lambda x, y, z: 1 + 0.2 * np.sin(2 * np.pi * (x + y + z)))
            errs.append((n, err))
            rate = math.log2(errs[-2][1] / err) if len(errs) > 1 else None
            out["runs"].append({"n": n, "order": order, "steps": steps, "l2_rho": err, "rate": rate,
                                "wall_s": wall})
            del s
            torch.cuda.empty_cache()
    print(json.dumps(out))


def main():
    args = parse()
    if args.err_steps is None:
        args.err_steps = 200 if args.order <= 3 else 100
    if args.sweep:
        run_sweep(args)
        return
    if args.ind_network:
        import torch
        import paper_1602_09079_gb300 as dgm
        dgm.load()
        print(json.dumps(_ind_network(dgm, torch, 3)))
        return
    if args.indicator:
        run_indicator(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
