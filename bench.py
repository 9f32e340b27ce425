"""Benchmark: cell-updates/s of the compact GKS with GENO reconstruction on the
2D 2048^2 periodic workload (16 random-phase density modes + 4 planar shocks,
Mach 1.5-3), mixed precision (FP32 reconstruction/flux, FP64 accumulation)
against FP64, with the density L1 and L-inf errors of mixed against FP64
after the same 20 and 100 CFL steps, beside the FP64 path's own divergence
from an input perturbed at FP32 rounding size (the workload's shocks amplify
rounding-level differences; by 100 steps both are about 4e-4 in L1).

One JSON line on rank 0.  A step is one full two-stage step of every cell
(gks_step_cfl: device time step, stage 1, stage 2).  `value` is the mixed-
precision device-timed rate; `fp64` holds the FP64 path's; `e2e` is the same
metric through the C ABI with host buffers (state copied in from pinned host
memory and read back every step).  `--impl reference` times the oracle (the
plain CPU implementation) on the host cores instead.

Rooflines: algorithmic flops per unit from the oracle's operation count
(tests/golden/flop_counts.json) against the pipe throughput the library's
probe kernels measure on this GPU (FP32 FMA, FP64 FMA).
Multi-GPU: replicas only (independent grids per rank, no exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 2048
SEED = 20463
CFL = 0.4
METRIC = "cell-updates/s and % HBM roofline, 2D 2048² mixed vs FP64, at stated L1 err"
WORKLOAD = "2D Euler 2048x2048 periodic, 16 random-phase density modes (k<=8) + 4 planar shocks Mach U[1.5,3], CFL 0.4"

# Algorithmic work per unit, from the oracle's operation count
# (tests/golden/flop_counts.json, written by tests/golden/make_flop_counts.py:
# the oracle's own arithmetic with common subexpressions shared and constants
# folded; flops = add/sub + mul + div, an FMA is 2; exp, erfc, sqrt and tanh
# are one op each and counted apart).
FLOPS = json.load(open(os.path.join(ROOT, "tests", "golden", "flop_counts.json")))


def _flops(key):
    return FLOPS[key]["flops"]


def _trans(key):
    return FLOPS[key]["transcendental"]


# face_flux_kernel, per face Gauss point: both interface states from the
# cubics (evaluation, admissibility) and the gas-kinetic flux
FACE_GP_2D = _flops("gks_point_2d") + _flops("face_states_gp_2d")
FACE_GP_2D_TRANS = _trans("gks_point_2d") + _trans("face_states_gp_2d")
# one cell advanced one full two-stage step (every kernel of the step)
CELL_UPDATE_2D = _flops("step_cell_update_2d")
CELL_UPDATE_3D = _flops("step_cell_update_3d")
# Navier-Stokes in 3D: the Euler step plus, per stage, the 12 face Gauss
# points of a cell with the viscous flux's extra work
CELL_UPDATE_3D_NS = CELL_UPDATE_3D + 2 * 12 * (_flops("gks_point_3d_ns") - _flops("gks_point_3d"))
# the WENO-Z / TENO weights change only the cubic of each (cell, variable)
CELL_UPDATE_2D_LIMITER = {lim: CELL_UPDATE_2D + 2 * 4 * (_flops(f"cubic_cell_var_2d_limiter{lim}")
                                                         - _flops("cubic_cell_var_2d_limiter0")) for lim in (2, 3)}
# 1D non-compact GENO + HLLC, one classical RK4 step (4 stages)
NC_CELL_UPDATE = {o: _flops(f"nc_step_cell_update_1d_order{o}") for o in (5, 6)}
# Executed flops of the face-flux kernel itself (ncu: 2 x FMA + ADD + MUL of
# the pipe, scalar and packed two-lane forms, per face Gauss point, on a 256^2 case whose index space is whole
# 128-item groups, so every point is evaluated exactly once; mean of the four
# launches of a step; the face-flux flop summary under profiles/).  The
# kernel uses closed forms where the oracle solves moment systems, so it
# executes fewer flops than the algorithmic count.
EXECUTED_FLOPS_PER_FACE_GP = {"mixed": 1523.8, "fp64": 1853.1}
# DRAM bytes (read + write) per launch of the face-flux kernel: the mean of
# the four launches of a 1-pass ncu capture at 1024^2 (coefficients 151 MB
# FP32 / 303 MB FP64, above L2): 200.5 MB mixed, 854.8 MB FP64, scaled to
# the 2048^2 launch by the Gauss points it processes.
TRAFFIC_PER_FLUX_LAUNCH = {"mixed": 200.51e6 * (2049 * 2048) / (1025 * 1024),
                           "fp64": 854.85e6 * (2049 * 2048) / (1025 * 1024)}
# Algorithmic HBM bytes per cell-update of the whole step (FP64 state,
# stage buffers, accumulator), 2D: 60 doubles.
BYTES_PER_CELL_UPDATE = 480.0


def measured_pipes(B):
    """Measured throughput of the arithmetic pipes (the library's probe
    kernels, CUDA-event timed): FP32 FMA (scalar and packed two-lane
    instructions) and FP64 FMA in TFLOP/s, the special-function unit in
    Tops/s.  The FP32 denominators take the larger of the two FP32 figures."""
    return {"ffma_tflops": B.pipe_probe(B.PIPE_FFMA, 4096) / 1e12,
            "ffma2_tflops": B.pipe_probe(B.PIPE_FFMA2, 4096) / 1e12,
            "dfma_tflops": B.pipe_probe(B.PIPE_DFMA, 64) / 1e12,
            "mufu_tops": B.pipe_probe(B.PIPE_MUFU, 256) / 1e12}


def alu_roofline(flops_per_unit, units_per_s, peak, kernel, unit_of_work, peak_source, traffic=None, nominal=None):
    """Roofline entry of a compute-bound kernel: algorithmic flops per unit x
    units per second against a measured pipe peak (TFLOP/s)."""
    ach = flops_per_unit * units_per_s / 1e12
    r = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
         "kernel": kernel, "flops_per_unit": flops_per_unit, "unit_of_work": unit_of_work,
         "numerator": "oracle op count (tests/golden/flop_counts.json)", "peak_source": peak_source}
    if nominal:
        r["frac_of_nominal"] = ach / nominal
    return r


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(n_sample: int = 256, steps: int = 2):
    """The oracle (FP64, OpenMP over all host cores) on a bounded sample of the
    workload: the same IC recipe on an n_sample^2 periodic grid."""
    import oracle
    from paper_2507_20461_gb300 import inputs as I

    W, G, h = I.fourier_shocks_2d(n_sample, SEED)
    cfg = oracle.make_cfg(2, (n_sample, n_sample), h, bc=0)
    t0 = time.perf_counter()
    for _ in range(steps):
        dt = CFL * h / oracle.max_wavespeed(cfg, W)
        r = oracle.step(cfg, dt, W, G)
        if r != 0:
            raise RuntimeError(f"oracle step failed: {r}")
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {
        "value": n_sample * n_sample * steps / el,
        "unit": "cell-updates/s",
        "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
        "kind": "oracle",
        "sample": f"{n_sample}x{n_sample} periodic grid of the same IC recipe, {steps} FP64 steps (wall {el:.1f} s)",
    }


def cpu_single_core(n_sample: int = 64, steps: int = 1):
    """The same oracle sample on one core: this script re-run with
    OMP_NUM_THREADS=1 (a fresh process, so the OpenMP runtime starts with one
    thread)."""
    import subprocess

    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(n_sample), "--cpu-steps", str(steps)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(f"single-core oracle run failed: {r.stderr[-400:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2507_20461_gb300 import inputs as I

    n_sample = 192
    W, G, h = I.fourier_shocks_2d(n_sample, SEED)
    cfg = oracle.make_cfg(2, (n_sample, n_sample), h, bc=0)
    for _ in range(args.warmup):
        oracle.step(cfg, CFL * h / oracle.max_wavespeed(cfg, W), W, G)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.step(cfg, CFL * h / oracle.max_wavespeed(cfg, W), W, G)
        if r != 0:
            raise RuntimeError(f"oracle step failed: {r}")
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    value = n_sample * n_sample * args.steps / el
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n_sample}x{n_sample} of the same IC recipe", "n": n_sample},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                          "sample": f"{n_sample}x{n_sample} periodic grid of the same IC recipe, one FP64 step per timed step"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_path(B, torch, W, G, h, precision, steps, warmup, dev, limiter=0, stage_kernels=0):
    """Device-timed steps of one precision; returns (ms/step, profile, final density)."""
    stream = torch.cuda.current_stream()
    s = B.Solver((N, N), bc=B.BC_PERIODIC, precision=precision, stream=stream, limiter=limiter,
                 stage_kernels=stage_kernels)
    Wd = torch.from_numpy(W).to(dev)
    Gd = torch.from_numpy(G).to(dev)
    s.set_state(Wd, Gd)
    s.step_cfl(CFL, warmup)
    torch.cuda.synchronize()
    s.profile(True, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_cfl(CFL, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prof = {k: s.profile_read(k) for k in (B.KC_RECON, B.KC_FACE, B.KC_UPDATE, B.KC_DT, B.KC_STAGE)}
    s.profile(False, False)
    st = s.status()
    s.get_state(Wd, Gd)
    rho = Wd[0].clone()
    s.close()
    return ms, prof, rho, st


def time_limiters(B, torch, W, G, h, steps, warmup, dev, ms_geno, ffma):
    """The WENO-Z and TENO weight variants (limiter 2, 3) on the headline
    workload, mixed precision, through the same timed path: they change only
    the per-cell reconstruction, so the face flux (the roofline kernel) is the
    headline's."""
    out = {"workload": "2D 2048^2 headline workload, mixed precision, limiter 2 (WENO-Z) / 3 (TENO)"}
    for name, lim in (("weno_z", 2), ("teno", 3)):
        ms, prof, _, st = time_path(B, torch, W, G, h, 1, steps, warmup, dev, limiter=lim)
        out[name] = {
            "value": N * N / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps, "status": st,
            "vs_geno_ms": ms / ms_geno,
            "kernel_ms": {nm: prof[k][1] / max(prof[k][0], 1) for k, nm in
                          ((B.KC_RECON, "cell_poly"), (B.KC_FACE, "face_flux"), (B.KC_UPDATE, "update"))},
            "roofline": alu_roofline(CELL_UPDATE_2D_LIMITER[lim], N * N / (ms * 1e-3), ffma, "whole step (all kernels)",
                                     "cell-update", "measured: FP32 FMA probe (scalar or packed, the larger)"),
        }
    return out


def time_noncompact(B, torch, steps, dev, dfma):
    """The 1D non-compact GENO schemes (order 5 and 6, HLLC flux, classical
    RK4; FP64) on 2^22 cells of the config-1 family (seeded two-state Riemann
    problem, transmissive), through gks_step_cfl.  Throughput and the split
    between the face kernel (reconstruction + HLLC) and the RK4 update."""
    import numpy as np

    from paper_2507_20461_gb300 import inputs as I

    n = 1 << 22
    W, G, h, _ = I.riemann_1d(n, seed=20461)
    out = {"workload": f"1D {n} cells, two-state Riemann IC (rho, p ~ U[0.1,1], u ~ U[-0.5,0.5]), transmissive, "
                       "CFL 0.4, FP64, one classical RK4 step per step"}
    stream = torch.cuda.current_stream()
    for order in (5, 6):
        s = B.Solver((n,), lo=[0.0], hi=[n * h], bc=B.BC_TRANSMISSIVE, precision=0, order=order, stream=stream)
        Wd = torch.from_numpy(np.ascontiguousarray(W)).to(dev)
        Gd = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
        s.set_state(Wd, Gd)
        s.step_cfl(CFL, 2)
        torch.cuda.synchronize()
        s.profile(True, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_cfl(CFL, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = {k: s.profile_read(k) for k in (B.KC_FACE, B.KC_UPDATE)}
        s.profile(False, False)
        st = s.status()
        s.close()
        out[f"order{order}"] = {
            "value": n / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps, "status": st,
            "kernel_ms_per_step": {"faces": prof[B.KC_FACE][1] / steps, "rk4_update": prof[B.KC_UPDATE][1] / steps},
            "roofline": alu_roofline(NC_CELL_UPDATE[order], n / (ms * 1e-3), dfma, "whole RK4 step (FP64)",
                                     "cell-update", "measured: DFMA probe"),
        }
    return out


def _guarded(fn, *a):
    """A secondary measurement: an exception becomes an error entry and
    leaves the rest of the line intact."""
    try:
        return fn(*a)
    except Exception as ex:  # noqa: BLE001
        return {"error": f"{type(ex).__name__}: {ex}"[:300]}


def time_e2e(B, torch, W, G, precision, steps, warmup, dev):
    """Same metric through the C ABI with host buffers: each step copies the
    state in from pinned host memory, steps, and reads the state back."""
    stream = torch.cuda.current_stream()
    s = B.Solver((N, N), bc=B.BC_PERIODIC, precision=precision, stream=stream)
    Wh = torch.from_numpy(W).pin_memory()
    Gh = torch.from_numpy(G).pin_memory()
    Wo = torch.empty_like(Wh).pin_memory()
    Go = torch.empty_like(Gh).pin_memory()
    for _ in range(warmup):
        s.set_state(Wh, Gh)
        s.step_cfl(CFL, 1)
        s.get_state(Wo, Go)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.set_state(Wh, Gh)
        s.step_cfl(CFL, 1)
        s.get_state(Wo, Go)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    s.close()
    nbytes = Wh.numel() * 8 + Gh.numel() * 8
    return N * N * steps / el, nbytes, nbytes


def aggregate(ws, ms_local, dist=None, device=None):
    """Max over ranks of the per-rank step times (replicas: each rank advances
    its own grid), so the whole-job rate is ws * cells / max time."""
    if ws == 1 or dist is None:
        return list(ms_local)
    import torch

    t = torch.tensor(list(ms_local), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def time_batch(B, torch, dev, ffma, total_steps=300, warm=3):
    """Config 4: 256 independent grids, sides log-uniform in [64, 1024], four-
    quadrant ICs (seed inputs.batch_seed(i): 20464 + i, the recorded grids
    redrawn), transmissive, CFL 0.4, the configuration's full 300 steps:
    `warm` steps (tuning, graph recording) and the remaining steps timed,
    mixed precision, graph replay.  The FP64 batch of the sampled grids runs
    the same 300 steps (each grid its own CFL time step, so the grids are
    independent of the rest), once from the input and once from the input
    perturbed at FP32 rounding size; density L1 / L-inf of mixed against FP64
    per sampled grid at step 300 (the worst grid is reported), with the
    perturbed FP64 run's beside it."""
    import numpy as np

    from paper_2507_20461_gb300 import inputs as I

    sides = I.batch_sizes(256, seed=20464)
    hs = [1.0 / n for n in sides]
    cells = sum(n * n for n in sides)
    states = [I.quadrants_2d(n, seed=I.batch_seed(g))[:2] for g, n in enumerate(sides)]
    out = {}
    rho = {}
    sample = (0, 1, 2, 100, 255)
    steps = total_steps - warm
    rng = np.random.default_rng(7)
    # runs: mixed (all grids, timed), FP64 and FP64 from the input perturbed
    # by a seeded relative 2^-24 (the sampled grids: the workload's own
    # sensitivity to rounding-size differences, beside mixed vs FP64)
    for run in ("mixed", "fp64", "fp64_perturbed"):
        prec = 1 if run == "mixed" else 0
        ids = list(range(len(sides))) if prec == 1 else list(sample)
        bt = B.Batch([sides[g] for g in ids], [sides[g] for g in ids], [hs[g] for g in ids],
                     bc=B.BC_TRANSMISSIVE, precision=prec)
        for k, g in enumerate(ids):
            W, G = states[g]
            if run == "fp64_perturbed":
                W = W * (1.0 + 2.0**-24 * rng.uniform(-1.0, 1.0, size=W.shape))
            bt.set_state(k, torch.from_numpy(np.ascontiguousarray(W)).to(dev), torch.from_numpy(G).to(dev))
        bt.run(CFL, warm)  # tuning + graph recording + warm steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        bt.run(CFL, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rho[run] = []
        for g in sample:
            Wd = torch.from_numpy(states[g][0]).to(dev)
            Gd = torch.from_numpy(states[g][1]).to(dev)
            bt.get_state(ids.index(g), Wd, Gd)
            rho[run].append(Wd[0].clone())
        gstat = bt.grid_status()
        if run == "mixed":
            out = {"value": cells / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps,
                   "total_steps": total_steps, "grids": 256, "cells": cells, "status": bt.status(),
                   "nonphysical_grids": {str(ids[k]): v for k, v in enumerate(gstat) if v},
                   "tuning": json.loads(bt.tuning() or "{}"),
                   "roofline": alu_roofline(CELL_UPDATE_2D, cells / (ms * 1e-3), ffma, "whole batched step",
                                            "cell-update", "measured: FP32 FMA probe (scalar or packed, the larger)")}
        elif run == "fp64":
            out["fp64_sampled_ms_per_step"] = ms
            out["fp64_status"] = bt.status()
            out["fp64_nonphysical_grids"] = {str(ids[k]): v for k, v in enumerate(gstat) if v}
        bt.close()
    spread = [(float((a - b).abs().mean()), float((a - b).abs().max()))
              for a, b in zip(rho["fp64_perturbed"], rho["fp64"])]
    errs = [(float((a - b).abs().mean()), float((a - b).abs().max())) for a, b in zip(rho["mixed"], rho["fp64"])]
    out[f"l1_density_mixed_vs_fp64_{total_steps}_steps"] = max(e[0] for e in errs)
    out[f"linf_density_mixed_vs_fp64_{total_steps}_steps"] = max(e[1] for e in errs)
    out[f"l1_density_fp64_perturbed_{total_steps}_steps"] = max(e[0] for e in spread)
    out["sampled_grids"] = {str(g): {"side": sides[g], "l1": e[0], "linf": e[1], "l1_fp64_perturbed": p[0],
                                     "linf_fp64_perturbed": p[1]} for g, e, p in zip(sample, errs, spread)}
    out["workload"] = ("256 grids, sides log-uniform [64,1024], four-quadrant ICs, transmissive, mixed precision, "
                       "graph replay, 300 steps")
    out["redrawn_grids"] = {str(g): I.batch_seed(g) for g in I.BATCH_REDRAWS}
    return out


def time_3d(B, torch, steps, dev, ffma):
    """Config 5: 3D 256^3 periodic solenoidal turbulence (rms Mach 0.6), mixed precision."""
    from paper_2507_20461_gb300 import inputs as I

    n = 256
    W, G, h = I.turbulence_3d(n, seed=20465)
    s = B.Solver((n, n, n), lo=[0, 0, 0], hi=[1, 1, 1], bc=B.BC_PERIODIC, precision=1)
    Wd = torch.from_numpy(W).to(dev)
    Gd = torch.from_numpy(G).to(dev)
    s.set_state(Wd, Gd)
    s.step_cfl(CFL, 2)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_cfl(CFL, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = s.status()
    s.close()
    return {"value": n**3 / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps, "status": st,
            "roofline": alu_roofline(CELL_UPDATE_3D, n**3 / (ms * 1e-3), ffma, "whole step (all kernels)",
                                     "cell-update", "measured: FP32 FMA probe (scalar or packed, the larger)"),
            "workload": "3D 256^3 periodic solenoidal velocity (E(k) ~ k^4 exp(-2(k/4)^2), rms Mach 0.6), mixed precision"}


def run_case_batch(count, steps):
    """A small run of the batched workload for ncu captures: `count` grids of
    the four-quadrant recipe (sides log-uniform in [64, 1024]), mixed
    precision, `steps` CFL steps (the first call tunes and records the graph)."""
    import numpy as np
    import torch

    from paper_2507_20461_gb300 import binding as B
    from paper_2507_20461_gb300 import inputs as I

    sides = I.batch_sizes(count, seed=I.BATCH_BASE_SEED)
    bt = B.Batch(sides, sides, [1.0 / n for n in sides], bc=B.BC_TRANSMISSIVE, precision=1)
    for g, n in enumerate(sides):
        W, G, h = I.quadrants_2d(n, seed=I.batch_seed(g))
        bt.set_state(g, torch.from_numpy(np.ascontiguousarray(W)).cuda(), torch.from_numpy(np.ascontiguousarray(G)).cuda())
    bt.run(CFL, 1)
    bt.run(CFL, steps)
    torch.cuda.synchronize()
    st = bt.status()
    bt.close()
    print(f"case batch grids={count} cells={sum(n * n for n in sides)} steps={steps + 1} status={st}")
    return 0 if st == 0 else 1


def run_case(n, precision, steps, stage_kernels=0):
    """A small run of the headline workload for ncu captures: the n^2
    periodic Fourier-mode + shock state, `steps` CFL steps through the C ABI
    (stage_kernels 1: the fused stage kernel)."""
    import numpy as np
    import torch

    from paper_2507_20461_gb300 import binding as B
    from paper_2507_20461_gb300 import inputs as I

    W, G, h = I.fourier_shocks_2d(n, SEED)
    s = B.Solver((n, n), bc=B.BC_PERIODIC, precision=precision, stage_kernels=stage_kernels)
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    Gd = torch.from_numpy(np.ascontiguousarray(G)).cuda()
    s.set_state(Wd, Gd)
    s.step_cfl(CFL, steps)
    torch.cuda.synchronize()
    st = s.status()
    s.close()
    print(f"case n={n} precision={precision} steps={steps} stage_kernels={stage_kernels} status={st}")
    return 0 if st == 0 else 1


def time_tgv(B, torch, steps, dev, ffma):
    """Navier-Stokes: the Taylor-Green vortex (u0 = 1, Ma 0.1, Re = 1600 with
    L0 = 2 pi, Prandtl 1) on 256^3 periodic cells of [-pi, pi]^3, mixed
    precision, through gks_step_cfl with the viscous time-step limit.  Its
    accuracy is checked by tests/test_gpu_ns.py (energy decay at Re 100)."""
    import math

    from paper_2507_20461_gb300 import inputs as I

    n = 256
    mu = 2 * math.pi / 1600.0
    W, G, h = I.taylor_green_3d(n)
    s = B.Solver((n, n, n), lo=[-math.pi] * 3, hi=[math.pi] * 3, bc=B.BC_PERIODIC, precision=1, mu=mu)
    Wd = torch.from_numpy(W).to(dev)
    Gd = torch.from_numpy(G).to(dev)
    s.set_state(Wd, Gd)
    s.step_cfl(CFL, 2)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_cfl(CFL, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = s.status()
    s.close()
    return {"value": n**3 / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms, "steps": steps, "status": st,
            "roofline": alu_roofline(CELL_UPDATE_3D_NS, n**3 / (ms * 1e-3), ffma, "whole step (all kernels)",
                                     "cell-update", "measured: FP32 FMA probe (scalar or packed, the larger)"),
            "workload": "3D Taylor-Green vortex 256^3, Navier-Stokes (Re 1600, Ma 0.1, Pr 1), mixed precision"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true", help="skip the batched and 3D workloads")
    ap.add_argument("--case", type=int, default=0, metavar="N",
                    help="profiling case: N^2 cells of the headline IC, --case-steps CFL steps, then exit (no JSON)")
    ap.add_argument("--case-precision", type=int, default=1, choices=[0, 1])
    ap.add_argument("--case-steps", type=int, default=2)
    ap.add_argument("--case-stage-kernels", type=int, default=0, choices=[0, 1])
    ap.add_argument("--case-batch", type=int, default=0, metavar="G",
                    help="ncu helper: a small batch of G grids of the batched recipe, then exit")
    ap.add_argument("--cpu-sample", type=int, default=0, metavar="N",
                    help="only time the oracle on an N^2 sample of the workload and print its JSON")
    ap.add_argument("--cpu-steps", type=int, default=1)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args.case, args.case_precision, args.case_steps, args.case_stage_kernels)
    if args.case_batch:
        return run_case_batch(args.case_batch, args.case_steps)
    if args.cpu_sample:
        print(json.dumps(cpu_baseline(args.cpu_sample, args.cpu_steps)))
        return 0

    import numpy as np
    import torch

    from paper_2507_20461_gb300 import binding as B
    from paper_2507_20461_gb300 import inputs as I

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    B.lib()

    W, G, h = I.fourier_shocks_2d(N, SEED)
    W = np.ascontiguousarray(W)
    G = np.ascontiguousarray(G)

    # FP64 path: fewer steps (about 10x slower), same warm-up rule
    steps64 = max(2, min(args.steps, 5))
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    pipes = measured_pipes(B)
    ms_mixed, prof_mixed, rho_mixed, st_mixed = time_path(B, torch, W, G, h, 1, args.steps, args.warmup, dev)
    ms_fused, prof_fused, _, st_fused = time_path(B, torch, W, G, h, 1, args.steps, args.warmup, dev, stage_kernels=1)
    ms_fp64, prof_fp64, rho_fp64, st_fp64 = time_path(B, torch, W, G, h, 0, steps64, args.warmup, dev)
    torch.cuda.synchronize()
    ms_mixed, ms_fused, ms_fp64 = aggregate(ws, [ms_mixed, ms_fused, ms_fp64], dist if ws > 1 else None, dev)
    clk = clocks.stop()

    # mixed vs FP64 on the same CFL steps (the FP64 path's time steps drive
    # every run), density L1 and L-inf after 20 and 100 steps; beside them the
    # workload's own sensitivity: the FP64 path from the input perturbed by a
    # seeded relative 2^-24 (the size of FP32 rounding)
    err_at = (20, 100)
    L1_STEPS = err_at[-1]
    rng = np.random.default_rng(7)
    Wp = W * (1.0 + 2.0**-24 * rng.uniform(-1.0, 1.0, size=W.shape))
    runs = []
    for prec, Win in ((0, W), (1, W), (0, Wp)):
        s_ = B.Solver((N, N), bc=B.BC_PERIODIC, precision=prec)
        Wd_, Gd_ = torch.from_numpy(np.ascontiguousarray(Win)).to(dev), torch.from_numpy(G).to(dev)
        s_.set_state(Wd_, Gd_)
        runs.append((s_, Wd_, Gd_))
    errors = {"mixed_vs_fp64": {}, "fp64_input_2^-24_vs_fp64": {}}
    for step in range(1, L1_STEPS + 1):
        dt = CFL * h / runs[0][0].max_wavespeed()
        for s_, _, _ in runs:
            s_.step(dt)
        if step in err_at:
            for s_, Wd_, Gd_ in runs:
                s_.get_state(Wd_, Gd_)
            for key, (_, Wd_, _) in zip(errors, runs[1:]):
                drho = (Wd_[0] - runs[0][1][0]).abs()
                errors[key][str(step)] = {"l1": float(drho.mean()), "linf": float(drho.max())}
    st_l1 = [s_.status() for s_, _, _ in runs]
    for s_, _, _ in runs:
        s_.close()
    del runs, Wp
    accuracy = {}
    for k in err_at:
        accuracy[f"l1_density_mixed_vs_fp64_{k}"] = errors["mixed_vs_fp64"][str(k)]["l1"]
        accuracy[f"linf_density_mixed_vs_fp64_{k}"] = errors["mixed_vs_fp64"][str(k)]["linf"]
        accuracy[f"l1_density_fp64_perturbed_{k}"] = errors["fp64_input_2^-24_vs_fp64"][str(k)]["l1"]
        accuracy[f"linf_density_fp64_perturbed_{k}"] = errors["fp64_input_2^-24_vs_fp64"][str(k)]["linf"]

    e2e_val, h2d, d2h = time_e2e(B, torch, W, G, 1, max(2, min(args.steps, 5)), 1, dev)
    ffma, dfma = max(pipes["ffma_tflops"], pipes["ffma2_tflops"]), pipes["dfma_tflops"]
    batch = None if args.headline_only else _guarded(time_batch, B, torch, dev, ffma)
    three_d = None if args.headline_only else _guarded(time_3d, B, torch, max(3, min(args.steps, 10)), dev, ffma)
    tgv = None if args.headline_only else _guarded(time_tgv, B, torch, max(3, min(args.steps, 10)), dev, ffma)
    limiters = None if args.headline_only else _guarded(
        time_limiters, B, torch, W, G, h, max(3, min(args.steps, 10)), args.warmup, dev, ms_mixed, ffma)
    noncompact = None if args.headline_only else _guarded(
        time_noncompact, B, torch, max(3, min(args.steps, 10)), dev, dfma)

    peaks, peak_src = _peaks()
    sm_clock = (clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    # nominal unit-count peaks, for context: 152 SMs x 128 FP32 lanes x 2 flop,
    # and 2 DFMA per SM per clock
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_nominal = nsm * 128 * 2 * sm_clock * 1e6 / 1e12
    fp64_nominal = nsm * 2 * 2 * sm_clock * 1e6 / 1e12

    # the dominant kernel: the face flux, one launch per direction; units per
    # launch = faces of one direction x 2 Gauss points
    units_per_launch = (N + 1) * N * 2
    n_face, t_face = prof_mixed[B.KC_FACE]
    avg_face_ms = t_face / max(n_face, 1)
    n64, t64 = prof_fp64[B.KC_FACE]
    avg64 = t64 / max(n64, 1)
    roof = alu_roofline(FACE_GP_2D, units_per_launch / (avg_face_ms * 1e-3), ffma, "face_flux_kernel<float,2,D,true>",
                        "face Gauss point", "measured: FP32 FMA probe (scalar or packed, the larger)", TRAFFIC_PER_FLUX_LAUNCH["mixed"], fp32_nominal)
    roof["transcendentals_per_unit"] = FACE_GP_2D_TRANS
    roof["launch_ms"] = avg_face_ms
    roof["units_per_launch"] = units_per_launch
    roof64 = alu_roofline(FACE_GP_2D, units_per_launch / (avg64 * 1e-3), dfma, "face_flux_kernel<double,2,D,true>",
                          "face Gauss point", "measured: DFMA probe", TRAFFIC_PER_FLUX_LAUNCH["fp64"], fp64_nominal)
    roof64["launch_ms"] = avg64
    for r, key in ((roof, "mixed"), (roof64, "fp64")):
        ex = EXECUTED_FLOPS_PER_FACE_GP[key]
        if ex:
            r["executed_flops_per_unit"] = ex
            r["frac_executed"] = r["frac"] * ex / FACE_GP_2D
    # the fused stage kernel: units per launch = cells (one stage of each)
    n_st, t_st = prof_fused[B.KC_STAGE]
    avg_stage_ms = t_st / max(n_st, 1)
    fused = {"value": ws * N * N / (ms_fused * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms_fused,
             "stage_launch_ms": avg_stage_ms, "status": st_fused, "vs_three_kernel_ms": ms_fused / ms_mixed,
             "roofline": alu_roofline(CELL_UPDATE_2D / 2, N * N / (avg_stage_ms * 1e-3), ffma,
                                      "fused2d_stage_kernel", "cell-stage", "measured: FP32 FMA probe (scalar or packed, the larger)")}

    launches_per_step = 1 + 1 + 2 * (1 + 2 + 1)  # wavespeed, dt, 2 x (poly, 2 face dirs, update)
    value = ws * N * N / (ms_mixed * 1e-3)
    value64 = ws * N * N / (ms_fp64 * 1e-3)
    hbm_frac = BYTES_PER_CELL_UPDATE * value / ws / (peaks.get("hbm_gbs", 6800.0) * 1e9)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        one = cpu_single_core()
        cpu["single_core"] = {"value": one["value"], "unit": one["unit"], "cores": one["cores"], "sample": one["sample"]}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_mixed,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "n": N,
            "precision": "mixed (FP32 reconstruction/flux, FP64 accumulation)",
            "l2": "inputs larger than L2 (state 403 MB per copy)",
            "parallelism": f"replicas x{ws}",
        },
        "fp64": {"value": value64, "ms_per_step": ms_fp64, "steps": steps64, "roofline": roof64,
                 "whole_step_roofline": alu_roofline(CELL_UPDATE_2D, value64 / ws, dfma, "whole step (all kernels)",
                                                     "cell-update", "measured: DFMA probe")},
        **accuracy,
        "density_errors": errors,
        "hbm_roofline_frac": hbm_frac,
        "roofline": roof,
        "whole_step_roofline": alu_roofline(CELL_UPDATE_2D, value / ws, ffma, "whole step (all kernels)",
                                            "cell-update", "measured: FP32 FMA probe (scalar or packed, the larger)"),
        "measured_pipes": pipes,
        "kernel_ms": {name: prof_mixed[k][1] / max(prof_mixed[k][0], 1) for k, name in
                      ((B.KC_RECON, "cell_poly"), (B.KC_FACE, "face_flux"), (B.KC_UPDATE, "update"), (B.KC_DT, "dt"))},
        "fused_stage_kernel": fused,
        "status": {"mixed": st_mixed, "fp64": st_fp64, "error_run": st_l1},
        "e2e": {"value": ws * e2e_val, "unit": "cell-updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "batched_256_grids": batch,
        "three_d_256": three_d,
        "navier_stokes_tgv_256": tgv,
        "limiter_variants_2048": limiters,
        "noncompact_1d": noncompact,
        "clocks": clk,
        "cpu_baseline": cpu,
        "peaks_source": peak_src,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
