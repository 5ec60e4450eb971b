#!/usr/bin/env python
"""Benchmark: tetrahedral-stencil FFT homogenization on GB300.

Workload (one "step"): a 256^3 periodic microstructure of seeded random
non-overlapping spheres (radius 8 voxels, volume fraction 0.30, isotropic
matrix E=1, nu=0.3), at four inclusion contrasts (E_i/E_m = 1e3, 1e-3, 1e6 as
the rigid surrogate, 0 = voids), each under the 6 unit macroscopic strains that
give the effective 6x6 stiffness: 24 solves, each to equilibrium error 1e-6 or
a budget of residual evaluations, with FP32 FFT/stencil/Green iterations and
FP64 residual sweeps, fields written.

Metric: voxel-iterations/s = sum over solves of N x (residual evaluations),
divided by the device time of the step (CUDA events, max over ranks).

``--impl reference`` times the CPU FP64 oracle instead (one Algorithm-1
iteration of the same 256^3 problem per step, on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

GRID = (256, 256, 256)
RADIUS = 8.0
FRACTION = 0.30
SEED = 1
CONTRASTS = [1e3, 1e-3, 1e6, 0.0]
NU = 0.3
TOL = 1e-6
# Residual evaluations allowed per solve inside a step.  At contrast 1e3 and
# the rigid surrogate the basic scheme needs thousands of evaluations on this
# microstructure, so a step runs every solve to err <= TOL or this budget,
# whichever comes first, and reports how many reached TOL.
BUDGET = 64
# DRAM bytes (read + write) per launch of the dominant kernel at the 256^3
# workload, from one ncu --set full capture of the current kernel (summarised
# with its command in profiles/iteration_kernels_256_fp32.md); set to None
# whenever that kernel changes until it is captured again.
NCU_TRAFFIC = {"xpass": 413.2e6}
METRIC = "voxel-iterations/s"
UNIT = "voxel-iter/s"


def unit_loads():
    out = []
    for J in range(6):
        e = np.zeros(6)
        e[J] = 1.0 if J < 3 else 0.5
        out.append(e)
    return out


def workload_config(precision_name):
    return {
        "workload": f"{GRID[0]}^3 random non-overlapping spheres R=8 f=0.30 (seed 1), isotropic nu=0.3, "
                    f"contrasts E_i/E_m in {CONTRASTS} (1e6 = rigid surrogate, 0 = void), 6 unit load cases each "
                    "-> C_eff, tol 1e-6",
        "grid": list(GRID),
        "solves_per_step": len(CONTRASTS) * 6,
        "precision": precision_name,
        "tol": TOL,
        "evaluation_budget_per_solve": BUDGET,
        "reference_medium": "paper Section 3.4 rule (k0 = a k_m + (1-a) k_i, same nu)",
        "l2": "inputs larger than L2: per solve the FP32 state + 2 work buffers are 3 x 203 MB",
    }


def make_inputs():
    ids, centres = synth.random_spheres(GRID, RADIUS, FRACTION, SEED)
    tables = [synth.two_phase_table(1.0, NU, c, NU) for c in CONTRASTS]
    return ids, tables


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.idx = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(kind, grid, refined=True):
    """Bytes each kernel class must move per launch (FP32 iteration kernels)."""
    n1, n2, n3 = grid
    N = n1 * n2 * n3
    nh = n1 // 2 + 1
    comp = n3 * n2 * nh * 8           # one FP32 complex half-spectrum component
    if kind == "xpass":               # real-space stencil: u in, ids, force out
        return 3 * N * 4 + 2 * N + 3 * N * 4
    if kind == "xpass_src":           # the same in a correction solve, which also reads the FP32 source
        return 3 * N * 4 + 2 * N + 3 * N * 4 + 3 * N * 4
    if kind == "x_inv":
        return 3 * comp + 3 * N * 4
    if kind == "x_fwd":
        return 3 * N * 4 + 3 * comp
    if kind in ("y_fwd", "y_inv"):
        return 2 * 3 * comp
    if kind == "z_green":
        return 4 * 3 * comp
    if kind == "resid64":
        return 3 * N * 8 + 2 * N + 3 * N * 4
    if kind == "fields":
        return 3 * N * 8 + 2 * N + 12 * N * 8
    return None


def cpu_sample(ids, table, workers=None):
    """One Algorithm-1 iteration of the oracle (evaluation + update) on the host."""
    from oracle import tetra as T

    grid = (ids.shape[2], ids.shape[1], ids.shape[0])
    mat = T.Material(ids, table)
    lam0 = T.c0_alpha_rule(table)
    D = T.D_of_q(grid)
    Om = T.green(D, lam0, grid)
    u = np.zeros((3, grid[2], grid[1], grid[0] // 2 + 1), dtype=np.complex128)
    E = T.unit_load(0)

    def one():
        nonlocal u
        t0 = time.perf_counter()
        _, _, _, _, f, L2, sm = T.evaluate(u, D, mat, E, grid, workers)
        u = u - np.einsum("jk...,k...->j...", Om, f)
        return time.perf_counter() - t0

    return one


def combine_over_ranks(ms, iters, device, world):
    """Replicas: the job's time is the slowest rank's, its work the sum of all ranks'."""
    if world <= 1:
        return float(ms), float(iters)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], device=device, dtype=torch.float64)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(t.item()), float(it.item())


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    ids, tables = make_inputs()
    cores = os.cpu_count() or 1
    step = cpu_sample(ids, tables[0], workers=cores)
    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    N = int(np.prod(GRID))
    total = sum(times)
    value = N * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config("oracle FP64 (scipy.fft), one Algorithm-1 iteration per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one Algorithm-1 iteration (evaluation + update) of the 256^3 "
                                   "contrast-1e3 E11 solve per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2405_11168_gb300 import hs

    hs.load()
    ids, tables = make_inputs()
    N = int(np.prod(GRID))
    ids_dev = torch.from_numpy(ids).to(dev)
    stream = torch.cuda.current_stream(dev)
    prec = hs.HS_FP32_REFINED
    solvers = [hs.Solver(ids_dev, t, precision=prec, device=dev, stream=stream) for t in tables]
    loads = unit_loads()
    shp = (6, GRID[2], GRID[1], GRID[0])
    eps_buf = torch.empty(shp, dtype=torch.float64, device=dev)
    sig_buf = torch.empty(shp, dtype=torch.float64, device=dev)

    import ctypes

    conv_log = []

    def solve_one(s, E):
        E = np.ascontiguousarray(E)
        sig_eff = np.zeros(6)
        it = ctypes.c_int()
        err = ctypes.c_double()
        st = s.lib.hs_solve(s.ctx, hs._dp(E), TOL, BUDGET, ctypes.c_void_p(eps_buf.data_ptr()),
                            ctypes.c_void_p(sig_buf.data_ptr()), hs._dp(sig_eff), ctypes.byref(it),
                            ctypes.byref(err))
        if st < 0:
            raise RuntimeError(f"solve failed: status {st}, err {err.value}")
        conv_log.append((st == hs.HS_OK, err.value))
        return it.value, sig_eff

    def step():
        iters = 0
        C = []
        for s in solvers:
            Ceff = np.zeros((6, 6))
            for J, E in enumerate(loads):
                k, se = solve_one(s, E)
                iters += k
                Ceff[:, J] = se
            C.append(Ceff)
        return iters, C

    for _ in range(args.warmup):
        step()
    for s in solvers:
        s.profile_read()
        s.profile(True)
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    conv_log.clear()
    ev0.record(stream)
    total_iters = 0
    for _ in range(args.steps):
        k, C = step()
        total_iters += k
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    timed_conv = list(conv_log)
    ms = ev0.elapsed_time(ev1)
    prof = {}
    for s in solvers:
        for k, (t, n) in s.profile_read().items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + t, b + n)
        s.profile(False)
    ms, total_iters_all = combine_over_ranks(ms, total_iters, dev, world)
    value = total_iters_all * N / (ms / 1e3)
    launches = int(sum(n for (_, n) in prof.values()))

    # dominant kernel roofline (time measured live with CUDA events on the launching stream)
    peak, peak_kind = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    roof = None
    if dom_n:
        per_launch_s = dom_ms / dom_n / 1e3
        b = algorithmic_bytes(dom_name, GRID)
        if dom_name in ("resid64", "fields"):
            # FP64 arithmetic bound: report against the FP64 ALU peak (1.25 TFLOP/s nominal)
            flops = FP64_FLOPS_PER_VOXEL * N
            ach = flops / per_launch_s / 1e12
            roof = {"bound": "alu", "kernel": dom_name, "achieved": ach, "peak": 1.25, "unit": "TFLOP/s",
                    "frac": ach / 1.25, "traffic": None, "peak_source": "nominal FP64 (GB300)"}
        else:
            ach = b / per_launch_s / 1e9
            traffic = NCU_TRAFFIC.get(dom_name) if tuple(GRID) == (256, 256, 256) else None
            roof = {"bound": "hbm", "kernel": dom_name, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs"}
    breakdown = {k: {"ms": round(t, 3), "launches": n,
                     "ms_per_launch": round(t / n, 4) if n else None,
                     "gbs": (round(algorithmic_bytes(k, GRID) / (t / n / 1e3) / 1e9, 1)
                             if n and algorithmic_bytes(k, GRID) else None)}
                 for k, (t, n) in prof.items() if n}

    # end to end: host ids in, C_eff out, through the C ABI each step
    e2e = None
    if not args.skip_e2e:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(args.steps):
            for t in tables:
                s = hs.Solver(ids, t, precision=prec, device=dev, stream=stream)
                for E in loads:
                    k, se = solve_one(s, E)
                    e_iters += k
                s.close()
                del s
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": e_iters * N / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(len(tables) * (ids.nbytes + 2 * 36 * 8)),
               "d2h_bytes_per_step": int(len(tables) * 6 * 6 * 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        one = cpu_sample(ids, tables[0], workers=cores)
        t = one()
        cpu = {"value": N / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one Algorithm-1 iteration (evaluation + update) of the 256^3 contrast-1e3 E11 solve, "
                         f"{t:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config("FP32 iterations + FP64 residual sweeps"),
                           parallelism=f"replicas x{world}"),
            "iterations_per_step": total_iters / args.steps,
            "solves_converged": f"{sum(c for c, _ in timed_conv)}/{len(timed_conv)}",
            "final_err_max": max(e for _, e in timed_conv),
            "roofline": roof, "kernels": breakdown, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# FP64 operations per voxel of the real-space residual sweep (isotropic phases):
# 2 tetrahedra x (gradient 3x6 adds + 3 x 3 scalings + 9 adds/doublings for the
# engineering strain, constitutive 12, adjoint 3 x (3 + 8)) + 8 x 3 accumulations
# + 3 FMA for |F|^2 + 6 stress sums.
FP64_FLOPS_PER_VOXEL = 2 * (18 + 9 + 9 + 12 + 33) + 24 + 6 + 6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--grid", type=int, default=256, help="cubic grid size (profiling runs use smaller cases)")
    ap.add_argument("--ncontrast", type=int, default=4, help="use the first k contrasts (profiling runs)")
    args = ap.parse_args()
    global GRID, CONTRASTS
    GRID = (args.grid,) * 3
    CONTRASTS = CONTRASTS[: max(1, min(4, args.ncontrast))]
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
