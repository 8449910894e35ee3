"""Benchmark: time steps/s of the immersed-boundary projection step on one
GB300, plus pressure-solve ms (FP64 multigrid vs FP32-inner defect
correction at equal 1e-10 residual) and the fine-level sweep's roofline.

Workload (default): 1024 x 1024 unit box, 64 seeded non-overlapping drops,
radii U[0.01, 0.03], 256 markers each (16384), density ratio 1000, viscosity
ratio 100, sigma = 1, irrotational spreading, B-spline relocation every 10
steps, pressure solved to ||r||/||b|| <= 1e-10 from the previous pressure.
A step = one ns_step (all stages of the time step).  L2 is flushed (256 MiB
write) before every timed step, outside the step's events.

--impl reference times the plain FP64 CPU oracle (its OpenMP build, all host
cores) on the same workload (each step one oracle time step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = ("pressure-solve ms & steps/s, FP64 MG vs mixed/NN-start at equal residual; %HBM")
SOLVERS = {0: "FP64 V(2,2)",
           1: "FP32 V(2,2) in FP64 defect correction",
           2: "FP32 V(2,2), two per FP64 residual, in FP64 defect correction"}
WORKLOADS = {
    "multidrop1024": dict(n=1024, kind="multi"),
    "multidrop512": dict(n=512, kind="multi16"),
    "multidrop2048": dict(n=2048, kind="multi"),
    "oscillating256": dict(n=256, kind="osc"),
    "static64": dict(n=64, kind="static"),
    "freefall_axi": dict(n=256, kind="freefall"),
}


def make_markers(name, seed_offset=0):
    wl = WORKLOADS[name]
    if wl["kind"] == "multi":
        return W.multidrop(wl["n"], seed=1811 + seed_offset)
    if wl["kind"] == "multi16":  # a quarter of the 1024^2 case, drops of the same size in cells
        return W.multidrop(wl["n"], ndrops=16, rmin=0.02, rmax=0.06, seed=1811 + seed_offset)
    if wl["kind"] == "osc":
        return W.oscillating_drop(seed=1808 + seed_offset)
    if wl["kind"] == "freefall":
        return W.freefall_axi()[0]
    return W.static_drop(wl["n"], 0.25, 128)


def problem(name):
    """Grid, physical constants and time step of a workload: (nx, ny, Config
    keyword arguments shared by the library and the oracle, dt).  Planar
    workloads: unit box, density ratio 1000, viscosity ratio 100, sigma 1.
    freefall_axi: the axisymmetric water drop in air (SI units) under gravity
    in the non-inertial frame."""
    if WORKLOADS[name]["kind"] == "freefall":
        _, c = W.freefall_axi()
        kw = dict(h=c["h"], rho_l=c["rho_l"], rho_g=c["rho_g"], mu_l=c["mu_l"], mu_g=c["mu_g"],
                  sigma=c["sigma"], gy=-c["g"], axisym=1, frame=1)
        dt = W.capillary_dt(c["h"], c["rho_l"], c["rho_g"], c["sigma"], c["mu_l"], c["mu_g"])
        return c["nx"], c["ny"], kw, dt
    n = WORKLOADS[name]["n"]
    return n, n, dict(h=1.0 / n), W.capillary_dt(1.0 / n, 1.0, 1e-3, 1.0, 1e-2, 1e-4)


def max_over_ranks(x: float) -> float:
    """Max of a host float over the ranks of the default process group (the
    identity when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def source_sha(rel, name):
    """Hash of the source file that holds kernel `name`: a recorded profile
    figure stays valid only while nothing in that file (the kernel, the
    device functions it inlines, its tile constants) has changed."""
    import hashlib
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def traffic_per_launch(kernel, cells):
    """DRAM bytes (read + write) of one launch over `cells` cells, from the
    per-cell figure of an ncu capture recorded in profiles/traffic.json; None
    when the kernel's source file has changed since that capture."""
    try:
        with open(TRAFFIC) as f:
            rec = json.load(f)[kernel]
        if source_sha(rec["source"], rec["function"]) != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_cell"] * cells
    except (OSError, KeyError, ValueError):
        return None


def host_info():
    """Host cores and CPU model, read at run time."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "hardware", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def oracle_rate(name, openmp, precision=2, budget_s=0.0, max_steps=1, warmup=0):
    """Oracle time steps/s on workload `name`: serial build (one core) or the
    OpenMP build (all host cores, bit-identical results).  After `warmup`
    untimed steps, runs at least one step and then as many of `max_steps` as
    fit in `budget_s` seconds.  Returns (steps/s, seconds, steps, threads)."""
    import oracle as O
    O.set_threads(openmp)
    try:
        O.build(openmp=openmp)
        mk = make_markers(name)
        nx, ny, kw, dt = problem(name)
        cfg = O.Config(nx=nx, ny=ny, precision=precision, spread=1, relocate_every=10, **kw)
        st = O.init_state(cfg, mk.X, mk.Y, mk.drop_start)
        for _ in range(warmup):
            O.ns_step(cfg, st, dt)
        done, t = 0, 0.0
        while done < max_steps and (done == 0 or t < budget_s):
            t0 = time.perf_counter()
            O.ns_step(cfg, st, dt)
            t += time.perf_counter() - t0
            done += 1
        return done / t, t, done, O.threads()
    finally:
        O.set_threads(False)


FP64_OPS = os.path.join(ROOT, "profiles", "fp64_ops.json")


def fp64_record(kernel):
    """The ncu record of a kernel in profiles/fp64_ops.json: executed FP64
    operations per work unit (its DFMA, DADD and DMUL thread instructions,
    an FMA counted as two, over its units) and the FP64 pipe's instruction
    rate (% of peak) in that capture; None when the kernel's source has
    changed since."""
    try:
        with open(FP64_OPS) as f:
            rec = json.load(f)[kernel]
        if source_sha(rec["source"], rec["function"]) != rec["source_sha256"]:
            return None
        return rec
    except (OSError, KeyError, ValueError, StopIteration):
        return None


def cpu_baseline(name):
    """One oracle time step of the workload on one core, then the OpenMP
    build on all host cores (the reported baseline is the faster one)."""
    info = host_info()
    v1, t1, _, _ = oracle_rate(name, False)
    try:
        vm, tm, _, thr = oracle_rate(name, True)
    except Exception as e:  # no OpenMP toolchain on this host
        vm, tm, thr = None, None, None
        info["openmp_error"] = str(e)[:200]
    best = (vm, thr, tm) if vm is not None and vm > v1 else (v1, 1, t1)
    return {"value": best[0], "unit": "steps/s", "cores": best[1], "kind": "oracle",
            "sample": f"1 oracle time step of {name} per variant "
                      f"(serial {t1:.1f} s" + (f", OpenMP {tm:.1f} s on {thr} threads)" if vm else ")"),
            "variants": {"serial": {"value": v1, "cores": 1, "seconds": t1},
                         "openmp": None if vm is None else {"value": vm, "cores": thr, "seconds": tm}},
            "build": "gcc -O3 -ffp-contract=off (+ -fopenmp)", **info}


def run_reference(args):
    """The oracle timed as it stands on the host cores (its OpenMP build, all
    cores; bit-identical to the serial one): W untimed warm-up steps, then as
    many of the K requested oracle time steps as fit in a 60 s budget (at
    least one); the per-step rate is the metric and `steps` is the number
    actually timed.  Rank 0 only."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    name = args.workload
    nx, ny, kw, dt = problem(name)
    info = host_info()
    try:
        value, t, done, thr = oracle_rate(name, True, args.precision, 60.0, args.steps,
                                          args.warmup)
    except Exception:
        value, t, done, thr = oracle_rate(name, False, args.precision, 60.0, args.steps,
                                          args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if args.precision >= 1 else "f64",
        "data": "synthetic",
        "config": {"workload": name, "nx": nx, "ny": ny, "solver": SOLVERS[args.precision],
                   "tol": 1e-10},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": thr, "kind": "oracle",
                         "sample": f"{done} of the {args.steps} requested oracle time steps of "
                                   f"{name} (60 s budget, {thr} threads)", **info},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# Algorithmic work per cell of the fused FP64 V(2,2) kernels (pre-scaled
# stencil; restricted residual from the red-black residual identity).
# Bytes: sweeps + residual + restriction read p, bt, the 4 weights (48),
# beta_x, beta_y (16), the coarse 1/diag (2), write p (8) and the coarse rc,
# btc, e (6); prolongation + sweeps read p, bt, the weights (48) and the
# coarse correction (2), write p (8).  FP64 operations (an FMA counted as
# two): a sweep 8 a cell; the residual 7 per red cell plus a subtraction per
# black cell, the restriction and pre-scaling 4 per coarse cell (5); the
# prolongation 7.
FP64_RESTRICT = {"bytes": 80.0, "flops": 2 * 8.0 + 5.0}
FP64_PROLONG = {"bytes": 58.0, "flops": 2 * 8.0 + 7.0}
# Per fine cell and V(2,2) cycle: the fully fused minimum of compulsory FP64
# traffic (84 B per level cell x 4/3 levels) and the per-kernel (unfused) accounting (212 B x 4/3); FP64
# operations of the FP64 cycle: (4 sweeps x 8 + 5 + 7) x 4/3 + the fine
# residual norm of the convergence test (15).
VCYCLE_BYTES_FUSED, VCYCLE_BYTES_UNFUSED = 112.0, 283.0
VCYCLE_FP64_FLOPS = (4 * 8.0 + 5.0 + 7.0) * 4.0 / 3.0 + 15.0


def timed_solve(torch, ctx, stream, flush, b, prec, start=None, reps=5, warm=3):
    """Median CUDA-event time of a cold (or given-start) solve to 1e-10
    through the solve graph; L2 flushed before each."""
    times, cyc, rr = [], None, None
    ny, nx = b.shape
    for rep in range(warm + reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p = start() if start is not None else torch.zeros((ny, nx), dtype=torch.float64,
                                                          device="cuda")
        st, cyc, rr = ctx.mg_solve(b, p, prec, 1e-10, 200)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= warm:
            times.append(e0.elapsed_time(e1))
    return {"ms": statistics.median(times), "cycles": cyc, "relres": rr}


def per_vcycle(entry, cells, pk, fp64_peak, fp64):
    """Per-V-cycle time and effective bandwidth (the fused 112 and the unfused
    283 B per fine cell) of a solve entry; FP64 cycles also against the FP64 peak."""
    us = 1e3 * entry["ms"] / max(entry["cycles"], 1)
    out = {"us": us}
    for label, B in (("fused_112B", VCYCLE_BYTES_FUSED), ("unfused_283B", VCYCLE_BYTES_UNFUSED)):
        gbs = B * cells / (us * 1e-6) / 1e9
        out[label] = {"GB_s": gbs, "frac_hbm": gbs / pk["hbm_gbs"]}
    if fp64:
        tf = VCYCLE_FP64_FLOPS * cells / (us * 1e-6) / 1e12
        out["fp64"] = {"flops_per_cell": VCYCLE_FP64_FLOPS, "tflops": tf, "frac": tf / fp64_peak}
    return out


def solve_and_kernels(ib, torch, ctx, stream, flush, nx, ny, net, pk, fp64_peak):
    """Pressure solve alone on the context's last system, cold start: FP64,
    precision 1, precision 2, and precision 2 from the network (inference
    inside the timed region); per-V-cycle figures; the level-0 kernels timed
    back to back on this data with their rooflines."""
    b = ctx.get("b")
    cells = nx * ny
    solve = {}
    for prec, label in ((0, "fp64"), (1, "mixed"), (2, "mixed2")):
        solve[label] = timed_solve(torch, ctx, stream, flush, b, prec)
    if net is not None:
        rho = ctx.get("rho")
        solve["mixed_cnn"] = timed_solve(torch, ctx, stream, flush, b, 2,
                                         start=lambda: net.infer(b[None], rho[None])[0])
        solve["mixed_cnn"]["solver"] = "mixed2 (two FP32 V-cycles per FP64 residual)"
    solve["speedup_vs_fp64"] = {k: solve["fp64"]["ms"] / solve[k]["ms"]
                                for k in ("mixed", "mixed2", "mixed_cnn") if k in solve}
    solve["per_vcycle"] = {k: per_vcycle(solve[k], cells, pk, fp64_peak, k == "fp64")
                           for k in ("fp64", "mixed", "mixed2")}
    us32, c0 = ctx.bench_kernel(4, 50)
    us64, _ = ctx.bench_kernel(1, 50)
    usr, _ = ctx.bench_kernel(7, 50)
    usp, _ = ctx.bench_kernel(8, 50)
    usn, _ = ctx.bench_kernel(6, 50)

    def roof(us, work, label):
        gbs = work["bytes"] * c0 / (us * 1e-6) / 1e9
        tf = work["flops"] * c0 / (us * 1e-6) / 1e12
        return {"kernel": label, "avg_launch_us": us, "algorithmic_bytes_per_cell": work["bytes"],
                "GB_s": gbs, "frac_hbm": gbs / pk["hbm_gbs"], "fp64_flops_per_cell": work["flops"],
                "fp64_tflops": tf, "frac_fp64": tf / fp64_peak,
                "bound": "fp64" if tf / fp64_peak > gbs / pk["hbm_gbs"] else "hbm"}
    kernels = {"level0": {
        "cells": int(c0), "fp32_prolong_sweeps2_us": us32, "fp64_sweep_us": us64,
        "fp64_sweeps2_restrict": roof(usr, FP64_RESTRICT, "k_smooth2_f64<1> (two FP64 sweeps + "
                                      "residual + restriction)"),
        "fp64_prolong_sweeps2": roof(usp, FP64_PROLONG, "k_smooth2_f64<2> (prolongation + two "
                                     "FP64 sweeps)"),
        "fp64_residual_norm": roof(usn, {"bytes": 32.0 + 8.0, "flops": 15.0},
                                   "k_resnorm (FP64 residual, norm, FP32 copy)")},
        "timing": "50 back-to-back launches on the level's data, CUDA events on the "
                  "launching stream (1024^2 data is largely L2-resident; 2048^2 is not)"}
    return solve, kernels


def static_drop_report(ib, steps=100):
    """The Laplace test of Section 5.1: the 64^2 static drop (R = 0.25 centred, 128 equispaced
    markers, density ratio 1000, viscosity ratio 100, sigma 1, FP64 solve to
    1e-10) after `steps` time steps, with the conventional and the
    irrotational spreading, markers as placed (curvature exactly 1/R) and
    with B-spline relocation every 10 steps: the largest parasitic velocity
    and the pressure jump of Section 5.1 Eq. (sd_pres_diff) (mean inside
    r < R - 4h minus mean outside r > R + 4h) against sigma / R = 4."""
    n, R = 64, 0.25
    h = 1.0 / n
    mk = W.static_drop(n, R, 128)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    c = (np.arange(n) + 0.5) * h
    d = np.hypot(*np.meshgrid(c - 0.5, c - 0.5))
    inside, outside = d < R - 4 * h, d > R + 4 * h
    out = {"grid": n, "steps": steps, "dt": dt, "jump_exact": 1.0 / R}
    for spread, sname in ((0, "conventional"), (1, "irrotational")):
        for reloc in (0, 10):
            cfg = ib.Config(nx=n, ny=n, h=h, spread=spread, relocate_every=reloc, precision=0,
                            tol=1e-10, max_cycles=200)
            ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
            ctx.ns_step(dt, steps, 1)
            u, v, p = ctx.get_host("u"), ctx.get_host("v"), ctx.get_host("p")
            jump = float(p[inside].mean() - p[outside].mean())
            out[f"{sname}_relocate{reloc}"] = {
                "max_u": float(max(np.abs(u).max(), np.abs(v).max())), "jump": jump,
                "jump_rel_err": abs(jump - 1.0 / R) * R}
            ctx.close()
    return out


def coarsen_for(n, args):
    """Halvings of an n x n grid before network inference: the given
    --cnn-coarsen, or (-1) as many as bring it to the training grid."""
    if args.cnn_coarsen >= 0:
        return args.cnn_coarsen
    k = 0
    while (n >> (k + 1)) >= args.cnn_grid and (n >> (k + 1)) % 4 == 0:
        k += 1
    return k


def steps_rate(ctx, torch, stream, flush, dt, warm, K):
    """Device-timed steps/s of K steps (CUDA events per step, L2 flushed
    before each)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        ctx.ns_step(dt, 1, warm)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return K / (sum(a.elapsed_time(b) for a, b in ev) / 1e3)


def scale_pass(ib, torch, args, stream, flush, net, pk, fp64_peak):
    """The scale configuration's other grid (2048^2 by default): steps/s with
    precision 2 and with the FP64 solver, the pressure solves and the level-0
    kernels on its data (which does not fit in L2)."""
    name = args.scale_workload
    nx, ny, kw, dt = problem(name)
    mk = make_markers(name)
    out = {"workload": name, "nx": nx, "ny": ny, "drops": int(mk.ndrops), "markers": int(mk.M)}
    for prec, key in ((2, "steps_per_s"), (0, "fp64_steps_per_s")):
        cfg = ib.Config(nx=nx, ny=ny, precision=prec, spread=1, relocate_every=10, tol=1e-10,
                        max_cycles=200, **kw)
        c = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
        for _ in range(args.warmup):
            c.ns_step(dt, 1, args.warm)
        out[key] = steps_rate(c, torch, stream, flush, dt, args.warm, args.scale_steps)
        if prec == 2:
            # the roofline kernel's launches inside the steps, as in the main pass
            ib.profile_begin(ib.PROF_PROLONG32)
            for _ in range(args.scale_steps):
                flush.zero_()
                c.ns_step(dt, 1, args.warm)
            torch.cuda.synchronize()
            sw_ms, sw_n = ib.profile_end()
            if net is not None:
                net.set_coarsen(coarsen_for(nx, args))
            solve, kernels = solve_and_kernels(ib, torch, c, stream, flush, nx, ny, net, pk,
                                               fp64_peak)
            if net is not None:
                solve["mixed_cnn"]["inference_grid"] = nx >> coarsen_for(nx, args)
            out["pressure_solve_ms"] = solve
            out["kernels"] = kernels
            us32 = kernels["level0"]["fp32_prolong_sweeps2_us"]
            gbs = 37.0 * nx * ny / (us32 * 1e-6) / 1e9
            us_in = sw_ms / sw_n * 1e3 if sw_n else None
            gbs_in = 37.0 * nx * ny / (us_in * 1e-6) / 1e9 if us_in else None
            out["roofline_fp32_smoother"] = {
                "kernel": "k_smooth2_f32<2> (fine level)", "algorithmic_bytes_per_cell": 37.0,
                "in_step_avg_launch_us": us_in, "in_step_launches": sw_n, "GB_s": gbs_in,
                "frac_hbm": gbs_in / pk["hbm_gbs"] if gbs_in else None,
                "back_to_back_us": us32, "back_to_back_GB_s": gbs,
                "back_to_back_frac_hbm": gbs / pk["hbm_gbs"],
                "traffic": traffic_per_launch("k_smooth2_f32<2>", nx * ny)}
        c.close()
    return out


def run_ours(args):
    import torch

    import paper_1807_10504_gb300 as ib

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ib.lib()
    name = args.workload
    nx, ny, kw, dt = problem(name)
    axi = bool(kw.get("axisym"))
    if axi:
        args.no_cnn = True  # the network is trained for the planar equation
    h = kw["h"]
    mk = make_markers(name, seed_offset=rank)  # independent problem per rank
    cfg = ib.Config(nx=nx, ny=ny, precision=args.precision, spread=1, relocate_every=10,
                    tol=1e-10, max_cycles=200, **kw)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    if args.no_graphs:
        ctx.use_graphs(False)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        ctx.ns_step(dt, 1, args.warm)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    if args.ncu_cnn:
        # network inference on this step's system inside a profiler range
        net = ib.Net(seed=0)
        net.set_coarsen(coarsen_for(nx, args))
        net.set_tensor_path(args.cnn_tensor_path)
        b, rho = ctx.get("b"), ctx.get("rho")
        net.infer(b[None], rho[None])
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            net.infer(b[None], rho[None])
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        ctx.close()
        return 0

    if args.ncu:
        torch.cuda.profiler.start()
        for k in range(args.steps):
            ctx.ns_step(dt, 1, args.warm)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        ctx.close()
        return 0

    sweep_kind = ib.PROF_PROLONG32 if args.precision >= 1 else ib.PROF_SWEEP64
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    cycles = []
    barrier()
    clk = Clocks(local)
    l0 = ib.launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        c, _ = ctx.ns_step(dt, 1, args.warm)
        ev[k][1].record(stream)
        cycles.append(c)
    barrier()
    launches = ib.launch_count() - l0
    clocks = clk.stop()
    t_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev))
    value = ws * args.steps / (t_ms / 1e3)

    # the same K steps again with CUDA events around every launch of the
    # roofline's kernel (the fine-level FP32 prolongation + post-smoothing
    # launch; the FP64 smoother launches at precision 0; per-launch events
    # need one launch per kernel, so this pass runs without the solve graph):
    # the roofline's kernel time
    ib.profile_begin(sweep_kind)
    for k in range(args.steps):
        flush.zero_()
        ctx.ns_step(dt, 1, args.warm)
    barrier()
    sweep_ms, sweep_n = ib.profile_end()

    # where the step's time goes: the same K steps three more times, CUDA
    # events on the context stream around one part of every step (the
    # step's graphs replay as in the timed steps)
    phases = {}
    for key, kind in (("before_solve", ib.PROF_PRE), ("solve", ib.PROF_SOLVE),
                      ("after_solve", ib.PROF_POST)):
        ib.profile_begin(kind)
        for k in range(args.steps):
            flush.zero_()
            ctx.ns_step(dt, 1, args.warm)
        barrier()
        ms, n = ib.profile_end()
        phases[key] = ms / max(n, 1)
    phases["unit"] = "ms per step"

    pk, pk_kind = peaks()
    fp64_peak = ib.probe_fp64()  # TFLOP/s, FMA chains on every SM

    # the same workload with the FP64 multigrid as the step's solver
    fp64_rate = None
    if args.precision != 0:
        c64 = ib.Context(ib.Config(nx=nx, ny=ny, precision=0, spread=1, relocate_every=10,
                                   tol=1e-10, max_cycles=200, **kw), mk.X, mk.Y, mk.drop_start)
        for _ in range(args.warmup):
            c64.ns_step(dt, 1, args.warm)
        fp64_rate = steps_rate(c64, torch, stream, flush, dt, args.warm, args.steps)
        c64.close()

    # mixed precision from the learned warm start: a network trained here on
    # solver-generated 128^2 samples (its own kernels), inference inside the
    # timed region
    net, train, cnn_eval = None, None, None
    if not args.no_cnn:
        from paper_1807_10504_gb300 import warmstart as WS
        t0 = time.perf_counter()
        data = WS.generate(args.cnn_samples, n_cells=args.cnn_grid, seed=0)
        t_gen = time.perf_counter() - t0
        net = ib.Net(seed=0)
        net.set_tensor_path(args.cnn_tensor_path)
        losses = WS.train(net, data, steps=args.cnn_steps, batch=args.cnn_batch, lr=2e-3)
        del data
        train = {"samples": args.cnn_samples, "grid": args.cnn_grid, "steps": len(losses),
                 "batch": args.cnn_batch, "first_loss": float(np.mean(losses[:20])),
                 "final_loss": float(np.mean(losses[-20:])), "generate_s": t_gen,
                 "train_s": time.perf_counter() - t0 - t_gen}
        # the learned warm start's evaluation case: an unseen seeded 512^2
        # system with 8 drops, cold / previous-step / network starts to 1e-10
        net.set_coarsen(coarsen_for(512, args))
        cnn_eval = {"grid": 512, "drops": 8, "inference_grid": 512 >> coarsen_for(512, args)}
        for prec in (1, 2):
            cnn_eval[f"precision{prec}"] = WS.evaluate(net, n_cells=512, ndrops=8, seed=1810,
                                                      precision=prec)
        net.set_coarsen(coarsen_for(nx, args))

    solve, kernels = solve_and_kernels(ib, torch, ctx, stream, flush, nx, ny, net, pk, fp64_peak)
    if train is not None:
        solve["mixed_cnn"]["train"] = train
        solve["mixed_cnn"]["inference_grid"] = nx >> coarsen_for(nx, args)
    us32, cells = kernels["level0"]["fp32_prolong_sweeps2_us"], kernels["level0"]["cells"]
    us64 = kernels["level0"]["fp64_sweep_us"]
    usb, pairs = ctx.bench_kernel(2, 10)
    # per-level durations of the mixed cycle's kernels (same method)
    levels = []
    for lev in range(16):
        row = {"level": lev}
        try:  # the FP32 cycle's kernels (levels above its single-CTA tail)
            t_down, c_l = ctx.bench_kernel(3, 20, lev)
            row.update(cells=int(c_l), sweeps2_restrict_us=t_down,
                       prolong_sweeps2_us=ctx.bench_kernel(4, 20, lev)[0],
                       sweeps2_us=ctx.bench_kernel(0, 20, lev)[0])
        except ib.IBError:
            pass
        try:  # the FP64 cycle's fused kernels (levels above its tail)
            t_r, c_l = ctx.bench_kernel(7, 20, lev)
            row.update(cells=int(c_l), fp64_sweeps2_restrict_us=t_r,
                       fp64_prolong_sweeps2_us=ctx.bench_kernel(8, 20, lev)[0],
                       fp64_sweep_us=ctx.bench_kernel(1, 20, lev)[0])
        except ib.IBError:
            pass
        if len(row) == 1:
            break
        levels.append(row)
    t_tail, c_tail = ctx.bench_kernel(5, 20)
    t_res, _ = ctx.bench_kernel(6, 20)
    kernel_table = {"levels": levels, "fp32_tail_us": t_tail, "fp32_tail_first_level_cells": int(c_tail),
                    "fp64_residual_norm_us": t_res}
    # algorithmic bytes per fine cell.  FP32 prolongation + sweeps at level 0
    # (defect correction): read the FP32 iterate, b, 1/diag, beta_x, beta_y
    # (20) and the coarse correction (4 B per 4 cells), read and write the
    # FP64 iterate (16).  FP64 sweep on the pre-scaled stencil: read p, bt
    # (16) and the four weights (32), write p (8).
    B32, B64 = 37.0, 56.0
    ach64 = B64 * cells / (us64 * 1e-6) / 1e9
    roof64 = {"kernel": "k_rbgs_sweep_w (fine level, one FP64 red-black sweep)", "bound": "hbm",
              "achieved": ach64, "peak": pk["hbm_gbs"], "unit": "GB/s",
              "frac": ach64 / pk["hbm_gbs"], "traffic": traffic_per_launch("k_rbgs_sweep_w", cells),
              "peak_source": pk_kind, "avg_launch_us": us64, "algorithmic_bytes_per_cell": B64,
              "algorithmic_bytes": B64 * cells,
              "fp64": {"flops_per_cell": 8.0, "achieved_tflops": 8.0 * cells / (us64 * 1e-6) / 1e12,
                       "peak_tflops": fp64_peak,
                       "frac": 8.0 * cells / (us64 * 1e-6) / 1e12 / fp64_peak}}
    band = {"kernel": "k_band_area", "avg_launch_us": usb, "pairs": int(pairs),
            "ns_per_pair": 1e3 * usb / max(pairs, 1)}
    # the marker side and the predictor: FP64-bound kernels stated against
    # the FP64 peak with their executed FP64 operations per unit (ncu)
    marker_side = {}
    for key, op, unit in (("k_band_area", 2, "(cell, segment) pair"), ("k_predictor", 9, "face"),
                          ("k_spread_irrot", 10, "face")):
        try:
            us_k, units_k = (usb, pairs) if op == 2 else ctx.bench_kernel(op, 10)
        except ib.IBError:
            continue
        rec = fp64_record(key)
        ent = {"avg_launch_us": us_k, "units": int(units_k), "unit": unit, "bound": "fp64"}
        if rec is not None:
            # FP64 operations counted as flops; the pipe also issues FP64
            # compares, min/max and conversions, which the capture's pipe
            # rate includes
            tf = rec["fp64_flops_per_unit"] * units_k / (us_k * 1e-6) / 1e12
            ent.update(fp64_flops_per_unit=rec["fp64_flops_per_unit"], fp64_tflops=tf,
                       peak_tflops=fp64_peak, frac=tf / fp64_peak,
                       fp64_pipe_pct_ncu=rec["fp64_pipe_pct_ncu"],
                       dram_bytes_per_unit_ncu=rec["dram_bytes_per_unit"])
        marker_side[key] = ent

    # the scale configuration's larger grid: 2048^2, same drops per unit area
    scale = None
    if args.scale_workload and args.scale_workload != name:
        scale = scale_pass(ib, torch, args, stream, flush, net, pk, fp64_peak)
    if net is not None:
        del net

    # end to end through the C ABI with host buffers: markers in, pressure out
    Xh = torch.empty(ctx.M, dtype=torch.float64).pin_memory().numpy()
    Yh = torch.empty(ctx.M, dtype=torch.float64).pin_memory().numpy()
    ph = torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy()
    ctx.get_markers_host(Xh, Yh)
    e2e_steps = max(3, args.steps // 2)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        # one call per step: markers in, the step, pressure and markers out
        ctx.ns_step_io(dt, args.warm, Xh, Yh, ph, Xh, Yh)
    barrier()
    e2e_t = max_over_ranks(time.perf_counter() - t0)

    avg_sweep = sweep_ms / max(sweep_n, 1)
    # the roofline's time: the kernel's average launch inside the steps
    B = B32 if args.precision >= 1 else B64
    us_b2b = us32 if args.precision >= 1 else us64
    ach = B * cells / (avg_sweep * 1e-3) / 1e9 if sweep_n else None
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.precision >= 1 else "f64", "data": "synthetic",
        "config": {"workload": name, "nx": nx, "ny": ny, "drops": int(mk.ndrops),
                   "markers": int(mk.M),
                   "density_ratio": round(cfg.rho_l / cfg.rho_g, 2),
                   "viscosity_ratio": round(cfg.mu_l / cfg.mu_g, 2),
                   "geometry": "axisymmetric (r, z), non-inertial frame" if axi else "planar",
                   "spread": "irrotational", "relocate_every": 10, "tol": 1e-10,
                   "solver": SOLVERS[args.precision],
                   "warm_start": {0: "zero", 1: "previous pressure",
                                  3: "2 p^n - p^(n-1)"}[args.warm],
                   "l2": "flushed before each step (256 MiB)",
                   "mean_vcycles_per_step": statistics.mean(cycles)},
        "pressure_solve_ms": solve,
        "learned_warm_start_512": cnn_eval,
        "static_drop_64": static_drop_report(ib),
        "fp64_steps_per_s": fp64_rate,
        "fp64_peak_tflops": fp64_peak,
        "fp64_kernels": kernels,
        "clocks": clocks,
        "e2e": {"value": ws * e2e_steps / e2e_t, "unit": "steps/s",
                "h2d_bytes_per_step": int(2 * ctx.M * 8),
                "d2h_bytes_per_step": int(nx * ny * 8 + 2 * ctx.M * 8)},
        "gpu_launches": int(launches),
        "roofline": {"kernel": ("k_smooth2_f32<2> (fine level: prolongation + two FP32 red-black "
                                "sweeps + FP64 update)" if args.precision >= 1 else
                                "k_rbgs_sweep_w (fine level, one FP64 red-black sweep)"),
                     "bound": "hbm", "achieved": ach,
                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / pk["hbm_gbs"] if ach else None,
                     "traffic": traffic_per_launch("k_smooth2_f32<2>" if args.precision >= 1
                                                   else "k_rbgs_sweep_w", cells),
                     "peak_source": pk_kind,
                     "avg_launch_us": avg_sweep * 1e3, "launches": sweep_n,
                     "algorithmic_bytes_per_cell": B,
                     "algorithmic_bytes": B * cells,
                     "cells_per_launch": int(cells),
                     "timing": "every launch of the kernel in K steps (the timed steps "
                               "repeated without the solve graph), CUDA events around each "
                               "launch on the launching stream, L2 flushed before each step",
                     "back_to_back_us": us_b2b,
                     "back_to_back_frac": B * cells / (us_b2b * 1e-6) / 1e9 / pk["hbm_gbs"],
                     "back_to_back_timing": "50 back-to-back launches on the step's "
                                            "fine-level data (largely L2-resident at 1024^2)"},
        "step_phases": phases,
        "roofline_fp64_sweep": roof64,
        "band_strip_areas": band,
        "fp64_marker_side": marker_side,
        "mixed_cycle_kernels": kernel_table,
    }
    if scale is not None:
        line["scale"] = scale
        rs = scale.get("roofline_fp32_smoother")
        if args.precision >= 1 and rs and rs.get("GB_s"):
            # %HBM is quoted on the larger grid, whose level does not fit in
            # L2 (at 1024^2 the smoother's operands largely stay there): the
            # same kernel, the same in-step timing, on the scale pass's steps
            sc = scale["nx"] * scale["ny"]
            line["roofline_1024"] = line["roofline"]
            line["roofline"] = {
                "kernel": line["roofline_1024"]["kernel"], "workload": scale["workload"],
                "bound": "hbm", "achieved": rs["GB_s"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": rs["frac_hbm"], "traffic": rs["traffic"], "peak_source": pk_kind,
                "avg_launch_us": rs["in_step_avg_launch_us"], "launches": rs["in_step_launches"],
                "algorithmic_bytes_per_cell": B32, "algorithmic_bytes": B32 * sc,
                "cells_per_launch": int(sc),
                "timing": (f"every launch of the kernel in {args.scale_steps} time steps of the "
                           f"{scale['workload']} pass (repeated without the solve graph), CUDA "
                           "events around each launch on the launching stream, L2 flushed before "
                           "each step; the level's operands exceed L2"),
                "back_to_back_us": rs["back_to_back_us"],
                "back_to_back_frac": rs["back_to_back_frac_hbm"],
                "back_to_back_timing": "50 back-to-back launches on the pass's fine-level data"}
    if axi:
        # the drop's fall so far: every ns_step of this run advanced it by dt
        com, S, vf, wb = ctx.frame_state()
        nsteps = args.warmup + 2 * args.steps + e2e_steps
        line["frame"] = {"steps": nsteps, "dt_s": dt, "t_s": nsteps * dt,
                         "drop_velocity_m_s": vf, "drop_centre_m": com,
                         "release_acceleration_m_s2": -kw["gy"] * (cfg.rho_l - cfg.rho_g)
                                                      / (cfg.rho_l + 0.5 * cfg.rho_g)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="multidrop1024", choices=list(WORKLOADS))
    ap.add_argument("--precision", type=int, default=2, choices=[0, 1, 2])
    ap.add_argument("--warm", type=int, default=1, choices=[0, 1, 3],
                    help="pressure initial guess of each step: 0 zero, 1 previous pressure, "
                         "3 extrapolated from the previous two")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cnn", action="store_true", help="skip the learned warm start")
    ap.add_argument("--cnn-samples", type=int, default=1500)
    ap.add_argument("--cnn-grid", type=int, default=256,
                    help="grid of the solver-generated training samples")
    ap.add_argument("--cnn-steps", type=int, default=1500)
    ap.add_argument("--cnn-batch", type=int, default=8)
    ap.add_argument("--cnn-tensor-path", type=int, default=1, choices=[0, 1, 2],
                    help="forward convolutions: 0 mma.sync everywhere, 1 tcgen05 where faster, "
                         "2 tcgen05 wherever the width allows")
    ap.add_argument("--cnn-coarsen", type=int, default=-1,
                    help="run the network on the grid coarsened by 2^k (-1: down to the "
                         "training grid)")
    ap.add_argument("--scale-workload", default="multidrop2048",
                    help="second grid of the scale configuration measured in the same run "
                         "(empty to skip)")
    ap.add_argument("--scale-steps", type=int, default=10)
    ap.add_argument("--no-graphs", action="store_true",
                    help="solve with one launch per kernel (for kernel profilers)")
    ap.add_argument("--ncu-cnn", action="store_true",
                    help="after the warm-up steps, only network inference on the step's system "
                         "inside a CUDA profiler range (random weights); prints no JSON")
    ap.add_argument("--ncu", action="store_true",
                    help="only warm-up + timed steps, the timed steps inside a CUDA profiler "
                         "range (for ncu --profile-from-start off); prints no JSON")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
