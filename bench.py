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

Beside the metric the line carries, each from its own leg outside the timed
region: the iterations and final errors per contrast of the timed solves and the
oracle's own error at one solve's final state (``err_vs_oracle``); a timing of
one solve that runs the FP32 correction solves (``correction_solves``); the
256^3 microstructure itself solved to 1e-6 at contrasts 1e3, 1e-3 and voids
(``converged_256``, with the oracle's error at one final state); 18
solves at 64^3 served to equilibrium error <= 1e-6 in plain FP64 and in FP32 +
FP64 refinement (``converged``: solves/s, p50/p99, the oracle's error at the
served states); 64 RVEs of sizes 32^3..128^3 with their 6 load cases in one
batch against the same solves one by one (``batched``); and a Poisson-arrival
request stream through the serving runtime (``serving``).

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
# workload, from one ncu capture of the current kernel (its summary, with the
# command, is kept under profiles/); set to None whenever that kernel changes
# until it is captured again.
NCU_TRAFFIC = {"xpass": 410.7e6, "z_green": 777.0e6}
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


class TorchFFTPipeline:
    """Library comparison: the same basic-scheme iteration (Algorithm 1) written
    with torch.fft (cuFFT on a GPU) and torch elementwise operations, in the
    real-space stencil form the CUDA path uses.  Not part of the library: the
    bench times it beside the CUDA kernels.

    State: the corner-indexed displacement spectrum u(q), complex
    [3][N3][N2][N1/2+1].  One iteration: u(r) by an unnormalised inverse FFT;
    for each tetrahedron the unscaled differences 2 D_i u_j over its four
    corners (Eqs. DA1-DA2), the engineering strain E + deps^T, the stress
    lambda(r) : strain (Algorithm 1 step 3); the nodal force
    F_k = 1/4 sum_T sum_corners sum_i c_i sigma^T_ik (the adjoint of the
    stencil, Eq. der_E_dep_Q); L2 = sqrt(sum |F|^2 / N), err = L2 / ||<sigma>||
    (Eqs. L2-norm, tolerance); F(q) by a 1/N forward FFT and
    u(q) <- u(q) - 2 Omega(q) F(q) (Algorithm 1 step 5, 2 F(q) = f(q)), with
    Omega^-1 = (lambda0 + mu0) M + mu0 tr(M) I, M_jk = 2 Re(D_j conj D_k)
    for the isotropic reference medium, and Omega = 0 at q = 0 and q = (pi, pi, pi).

    Two isotropic phases (a 6x6 table per phase with C = 0 for a void);
    reference medium by the Section 3.4 rule (same nu as the matrix,
    k0 = a k_m + (1 - a) k_i, a = 0.55 if k_i < k_m else 0.45).
    """

    # corners of each tetrahedron as (shift (ox, oy, oz): corner index = voxel
    # index - shift, coefficients c_i of 2 D_i u = sum_corners c_i u(corner))
    TETRA = (
        (((0, 0, 0), (1, 1, 1)), ((0, 1, 1), (1, -1, -1)), ((1, 1, 0), (-1, -1, 1)), ((1, 0, 1), (-1, 1, -1))),
        (((0, 1, 0), (1, -1, 1)), ((0, 0, 1), (1, 1, -1)), ((1, 1, 1), (-1, -1, -1)), ((1, 0, 0), (-1, 1, 1))),
    )
    # Voigt index of the tensor component (i, k)
    VOIGT = ((0, 5, 4), (5, 1, 3), (4, 3, 2))

    def __init__(self, ids, table, device, dtype=None):
        import torch

        self.torch = torch
        self.dtype = dtype or torch.float32
        self.cdtype = torch.complex64 if self.dtype == torch.float32 else torch.complex128
        table = np.asarray(table, dtype=np.float64)
        n3, n2, n1 = ids.shape
        self.grid = (n1, n2, n3)
        self.N = n1 * n2 * n3
        lam = table[:, 0, 1]
        mu = table[:, 3, 3]
        idt = torch.as_tensor(np.ascontiguousarray(ids).astype(np.int64), device=device)
        self.lam = torch.as_tensor(lam, dtype=self.dtype, device=device)[idt]
        self.mu = torch.as_tensor(mu, dtype=self.dtype, device=device)[idt]
        # reference medium (Section 3.4 rule)
        k_m, k_i = lam[0] + 2 * mu[0] / 3, lam[1] + 2 * mu[1] / 3
        a = 0.55 if k_i < k_m else 0.45
        k0 = a * k_m + (1 - a) * k_i
        nu0 = lam[0] / (2 * (lam[0] + mu[0]))
        mu0 = 3 * k0 * (1 - 2 * nu0) / (2 * (1 + nu0))
        lam0 = k0 - 2 * mu0 / 3
        # Omega(q) in FP64, stored in the working precision: [3][3][N3][N2][N1/2+1]
        h1 = np.arange(n1 // 2 + 1)[None, None, :]
        h2 = np.arange(n2)[None, :, None]
        h3 = np.arange(n3)[:, None, None]
        q = (2 * np.pi * h1 / n1, 2 * np.pi * h2 / n2, 2 * np.pi * h3 / n3)
        D = np.zeros((3, n3, n2, n1 // 2 + 1), dtype=np.complex128)
        for shift, c in self.TETRA[0]:
            ph = np.exp(-1j * (shift[0] * q[0] + shift[1] * q[1] + shift[2] * q[2]))
            for i in range(3):
                D[i] = D[i] + 0.5 * c[i] * ph
        M = 2.0 * np.real(D[:, None] * np.conj(D[None, :]))
        Oi = (lam0 + mu0) * M + mu0 * np.trace(M)[None, None] * np.eye(3)[:, :, None, None, None]
        Oi = np.moveaxis(Oi, (0, 1), (-2, -1))
        sing = np.zeros(Oi.shape[:3], dtype=bool)
        sing[0, 0, 0] = True
        if n1 % 2 == 0 and n2 % 2 == 0 and n3 % 2 == 0:
            sing[n3 // 2, n2 // 2, n1 // 2] = True
        Oi[sing] = np.eye(3)
        Om = np.linalg.inv(Oi)
        Om[sing] = 0.0
        self.Om = torch.as_tensor(np.moveaxis(Om, (-2, -1), (0, 1)).copy(), dtype=self.dtype, device=device)
        self.uh = torch.zeros((3, n3, n2, n1 // 2 + 1), dtype=self.cdtype, device=device)
        self.C = [torch.tensor([c for _, c in tet], dtype=self.dtype, device=device) for tet in self.TETRA]

    def step(self, E):
        """One evaluation + update; returns (err, <sigma> Voigt)."""
        torch = self.torch
        n1, n2, n3 = self.grid
        Eeng = [float(E[i]) * (1.0 if i < 3 else 2.0) for i in range(6)]
        u = torch.fft.irfftn(self.uh, s=(n3, n2, n1), dim=(1, 2, 3), norm="forward")
        F = torch.zeros_like(u)
        ssum = torch.zeros(6, dtype=torch.float64, device=u.device)
        for tet, C in zip(self.TETRA, self.C):
            U = torch.stack([torch.roll(u, shifts=(sh[2], sh[1], sh[0]), dims=(1, 2, 3)) for sh, _ in tet])
            g = torch.einsum("vi,vj...->ij...", C, U)  # g[i][j] = 2 D_i u_j
            e = [Eeng[0] + 0.5 * g[0, 0], Eeng[1] + 0.5 * g[1, 1], Eeng[2] + 0.5 * g[2, 2],
                 Eeng[3] + 0.5 * (g[1, 2] + g[2, 1]), Eeng[4] + 0.5 * (g[0, 2] + g[2, 0]),
                 Eeng[5] + 0.5 * (g[0, 1] + g[1, 0])]
            del U, g
            lt = self.lam * (e[0] + e[1] + e[2])
            m2 = 2 * self.mu
            s = [lt + m2 * e[0], lt + m2 * e[1], lt + m2 * e[2], self.mu * e[3], self.mu * e[4], self.mu * e[5]]
            ssum += torch.stack([torch.sum(x, dtype=torch.float64) for x in s])
            S = torch.stack([s[self.VOIGT[i][k]] for i in range(3) for k in range(3)]).view((3, 3) + u.shape[1:])
            contrib = torch.einsum("vi,ik...->vk...", C, S)  # sum_i c_i sigma_ik per corner
            for v, (sh, _) in enumerate(tet):
                F += torch.roll(contrib[v], shifts=(-sh[2], -sh[1], -sh[0]), dims=(1, 2, 3))
        F *= 0.25
        l2 = torch.sqrt(torch.sum(F * F, dtype=torch.float64) / self.N)
        sm = 0.5 * ssum / self.N
        nrm = torch.sqrt(torch.sum(sm[:3] ** 2) + 2 * torch.sum(sm[3:] ** 2))
        Fh = torch.fft.rfftn(F, dim=(1, 2, 3), norm="forward")
        for j in range(3):
            self.uh[j] -= 2 * (self.Om[j, 0] * Fh[0] + self.Om[j, 1] * Fh[1] + self.Om[j, 2] * Fh[2])
        return l2 / nrm, sm


def time_torch_pipeline(ids, table, device, iters, warmup=2):
    """ms per iteration of TorchFFTPipeline on the device (CUDA events), the
    error after the timed iterations, and ms per iteration of its six FFTs alone."""
    import torch

    p = TorchFFTPipeline(ids, table, device)
    E = unit_loads()[0]
    for _ in range(warmup):
        p.step(E)
    stream = torch.cuda.current_stream(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    ev0.record(stream)
    for _ in range(iters):
        err, _ = p.step(E)
    ev1.record(stream)
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1) / iters
    last = float(err)
    # the six transforms of an iteration alone (3 components inverse + forward):
    # the floor of any iteration built on these library FFTs
    n1, n2, n3 = p.grid
    torch.cuda.synchronize(device)
    ev0.record(stream)
    for _ in range(iters):
        u = torch.fft.irfftn(p.uh, s=(n3, n2, n1), dim=(1, 2, 3), norm="forward")
        fh = torch.fft.rfftn(u, dim=(1, 2, 3), norm="forward")
    ev1.record(stream)
    torch.cuda.synchronize(device)
    fft_ms = ev0.elapsed_time(ev1) / iters
    del p, u, fh
    torch.cuda.empty_cache()
    return ms, last, fft_ms


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


def oracle_err_at(u_real, ids, table, E6):
    """The oracle's equilibrium error (Eqs. L2-norm, tolerance) and <sigma> at a real-space
    corner displacement (corner (l+1/2, m+1/2, n+1/2) at index (l, m, n)): Algorithm 1 steps
    1-4 evaluated once at that state, in FP64 on the host."""
    from oracle import tetra as T

    n3, n2, n1 = ids.shape
    grid = (n1, n2, n3)
    q1, q2, q3 = T.q_vectors(grid)
    u_q = T.ft(np.asarray(u_real, dtype=np.float64)) * np.exp(-0.5j * (q1 + q2 + q3))[None]
    _, _, _, _, _, L2, sm = T.evaluate(u_q, T.D_of_q(grid), T.Material(ids, table), T.strain_tensor_from_voigt(E6),
                                       grid)
    return float(L2 / np.sqrt(np.sum(sm ** 2))), T.voigt_from_tensor(sm)


def state_check(s, ids, table, E6, gpu_err, gpu_sig):
    """The oracle's error and <sigma> at a solver's final displacement against what the GPU reported."""
    err, sm = oracle_err_at(s.get_displacement().cpu().numpy(), ids, table, E6)
    return {"gpu_err": gpu_err, "oracle_err_at_gpu_state": err,
            "err_rel_diff": abs(err - gpu_err) / max(err, 1e-300),
            "sig_eff_rel_diff": float(np.max(np.abs(np.asarray(gpu_sig) - sm)) / np.max(np.abs(sm)))}


def per_contrast(log):
    """Iterations and final errors of logged solves, by contrast."""
    out = {}
    for c in sorted({x["contrast"] for x in log}, key=lambda v: -v):
        xs = [x for x in log if x["contrast"] == c]
        out[f"{c:g}"] = {"solves": len(xs), "converged": sum(x["status"] == 0 for x in xs),
                         "evaluations": sorted({x["iters"] for x in xs}),
                         "final_err_min": min(x["err"] for x in xs), "final_err_max": max(x["err"] for x in xs)}
    return out


def correction_leg(hs, ids_dev, table, dev, stream):
    """One 256^3 solve whose budget runs FP32 correction solves: the first FP32 solve and every
    correction solve get at most 40 evaluations, 200 in all, every launch timed."""
    s = hs.Solver(ids_dev, table, precision=hs.HS_FP32_REFINED, device=dev, stream=stream, inner_max=40)
    E = unit_loads()[0]
    s.solve(E, tol=TOL, max_iter=200, fields=False)
    s.profile_read()
    s.profile(1)
    out = s.solve(E, tol=TOL, max_iter=200, fields=False)
    prof = s.profile_read()
    s.profile(False)
    hist = s.err_history()
    s.close()
    # GB/s of the algorithmic bytes for the HBM-side kernels only (the FP64 sweep is FP64-pipe bound)
    kern = {k: {"ms_per_launch": round(t / n, 4), "launches": n,
                "gbs": (round(algorithmic_bytes(k, GRID) / (t / n / 1e3) / 1e9, 1)
                        if algorithmic_bytes(k, GRID) and k not in ("resid64", "fields") else None)}
            for k, (t, n) in prof.items() if n}
    return {"what": f"{GRID[0]}^3 contrast {CONTRASTS[0]:g} E11, inner_max 40, budget 200 evaluations, every launch "
                    "timed with CUDA events", "evaluations": out["iters"], "status": out["status"],
            "final_err": out["err"], "fp64_sweep_errs": [float(x) for x in hist[40:]][-8:], "kernels": kern}


def converged_256_leg(hs, ids, ids_dev, dev, stream):
    """The bench microstructure itself (256^3) solved to err <= 1e-6 in FP32 + FP64 refinement,
    E11, one solve per contrast 1e3, 1e-3 and voids (budget 20000 evaluations), timed with CUDA
    events; the oracle's error at the 1e-3 solve's final state; the rigid surrogate 1e6 with a
    budget of 2000 evaluations (its FP64 iteration stalls on random packings, see the design notes)."""
    import torch

    E = unit_loads()[0]
    rows = {}
    for c, budget in ((1e3, 20000), (1e-3, 20000), (0.0, 20000), (1e6, 2000)):
        table = synth.two_phase_table(1.0, NU, c, NU)
        s = hs.Solver(ids_dev, table, precision=hs.HS_FP32_REFINED, device=dev, stream=stream)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        o = s.solve(E, tol=TOL, max_iter=budget, fields=False)
        t1.record(stream)
        t1.synchronize()
        row = {"status": o["status"], "converged": o["status"] == hs.HS_OK, "evaluations": o["iters"],
               "final_err": o["err"], "s": t0.elapsed_time(t1) / 1e3, "budget": budget}
        if c == 1e-3:
            row["err_vs_oracle"] = state_check(s, ids, table, E, o["err"], o["sig_eff"])
        s.close()
        rows[f"{c:g}"] = row
    return {"what": f"{GRID[0]}^3 random spheres R=8 f=0.30 seed 1 (the timed workload), E11, FP32 + FP64 "
                    "refinement, tol 1e-6, one solve per contrast", "solves": rows}


CONV_GRID = (64, 64, 64)
CONV_CONTRASTS = [1e3, 1e-3, 0.0]


def converged_leg(hs, dev):
    """18 solves (64^3 random spheres R = 8, f = 0.30, seed 1; contrasts 1e3, 1e-3 and voids, 6 unit
    loads each) served to err <= 1e-6 through the resident serving runtime, in plain FP64 and in
    FP32 + FP64 refinement; the first pass creates the resident contexts, the second is timed.
    The oracle's own error at each contrast's E11 state is reported beside the GPU's.  The rigid
    surrogate 1e6 is run alone with a 3000-evaluation budget in both precisions."""
    from paper_2405_11168_gb300 import serve

    ids, _ = synth.random_spheres(CONV_GRID, RADIUS, FRACTION, SEED)
    N = int(np.prod(CONV_GRID))
    out = {"workload": f"{CONV_GRID[0]}^3 random spheres R=8 f=0.30 seed 1, contrasts {CONV_CONTRASTS}, "
                       "6 unit loads each (18 solves), tol 1e-6, 3 serving slots, resident contexts"}
    for name, prec in (("fp64", hs.HS_FP64), ("fp32_refined", hs.HS_FP32_REFINED)):
        tables = [synth.two_phase_table(1.0, NU, c, NU) for c in CONV_CONTRASTS]
        srv = serve.Server(budget_bytes=40 << 30, slots=3, device=dev)
        try:
            def reqs():
                return [serve.Request(ids=ids, table=t, loads=unit_loads(), precision=prec, tol=TOL, max_iter=20000,
                                      tag=c) for t, c in zip(tables, CONV_CONTRASTS)]
            serve.run_stream(srv, reqs(), 0.0)
            res, wall = serve.run_stream(srv, reqs(), 0.0)
        finally:
            srv.close()
        solves = sum(len(r.iters) for r in res)
        evals = sum(sum(r.iters) for r in res)
        row = {"solves_per_s": solves / wall, "solves": solves, "wall_s": wall,
               "converged": sum(int(st == hs.HS_OK) for r in res for st in r.status),
               "voxel_iter_per_s": evals * N / wall, "evaluations": {f"{r.tag:g}": r.iters for r in res},
               "final_err_max": max(max(r.errs) for r in res), **serve.latency_stats(res),
               "latency_is": "per request (6 solves), all 3 requests submitted at once", "err_vs_oracle": {}}
        for t, c in zip(tables, CONV_CONTRASTS):
            s = hs.Solver(ids, t, precision=prec, device=dev)
            o = s.solve(unit_loads()[0], tol=TOL, max_iter=20000, fields=False)
            row["err_vs_oracle"][f"{c:g}"] = state_check(s, ids, t, unit_loads()[0], o["err"], o["sig_eff"])
            s.close()
        rig = hs.Solver(ids, synth.two_phase_table(1.0, NU, 1e6, NU), precision=prec, device=dev)
        o = rig.solve(unit_loads()[0], tol=TOL, max_iter=3000, fields=False)
        rig.close()
        row["rigid_1e6_E11"] = {"status": o["status"], "evaluations": o["iters"], "final_err": o["err"]}
        out[name] = row
    out["refined_over_fp64_solves_per_s"] = out["fp32_refined"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


BATCH_SIZES = (32, 48, 64, 96, 128)


def batch_rves(n_rve=64, seed=4):
    """64 RVEs: sizes uniform over 32^3..128^3; half random spheres (R = 8, f = 0.30, contrast
    log-uniform in 1e-3..1e3), half 50-grain cubic Voronoi polycrystals (C11 = 168.4,
    C12 = 121.4, C44 = 75.4 rotated per grain)."""
    rng = np.random.default_rng(seed)
    rves = []
    for _ in range(n_rve):
        n = int(rng.choice(BATCH_SIZES))
        if rng.random() < 0.5:
            ids, _ = synth.random_spheres((n, n, n), RADIUS, FRACTION, int(rng.integers(1 << 30)))
            table = synth.two_phase_table(1.0, NU, float(10.0 ** rng.uniform(-3, 3)), NU)
        else:
            ids, _ = synth.voronoi_grains((n, n, n), 50, seed=int(rng.integers(1 << 30)))
            ids = ids.astype(np.uint8)
            table = synth.polycrystal_table(168.4, 121.4, 75.4, synth.random_rotations(50, seed=int(rng.integers(1 << 30))))
        rves.append((ids, table))
    return rves


def batched_leg(hs, dev, budget=200):
    """The 64 RVEs x 6 load cases (384 items) in one batch against the same 384 solves one by one
    (one resident solver per RVE), FP32 + FP64 refinement, tol 1e-6, the same evaluation budget per
    solve; the iterates are identical either way, so the two voxel-iteration rates compare the same
    work."""
    rves = batch_rves()
    item_rve = [r for r in range(len(rves)) for _ in range(6)]
    E = np.array([e for _ in rves for e in unit_loads()])
    Ns = np.array([rves[r][0].size for r in item_rve], dtype=np.float64)
    stream = torch_stream(dev)
    b = hs.Batch(rves, item_rve, precision=hs.HS_FP32_REFINED, device=dev, stream=stream, autotune=True)
    nclass, _ = b.classes()
    b.solve(E, tol=TOL, max_iter=budget)
    b.launches()
    t0 = cuda_time(dev, stream)
    ob = b.solve(E, tol=TOL, max_iter=budget)
    tb = cuda_time(dev, stream) - t0
    launches_b = b.launches()
    b.close()
    del b
    solvers = [hs.Solver(ids, t, precision=hs.HS_FP32_REFINED, device=dev, stream=stream) for ids, t in rves]
    for s in solvers:
        s.solve(unit_loads()[0], tol=TOL, max_iter=budget, fields=False)
    t0 = cuda_time(dev, stream)
    it1 = []
    for i, r in enumerate(item_rve):
        it1.append(solvers[r].solve(E[i], tol=TOL, max_iter=budget, fields=False)["iters"])
    t1 = cuda_time(dev, stream) - t0
    for s in solvers:
        s.close()
    vb = float(np.sum(ob["iters"] * Ns)) / tb
    v1 = float(np.sum(np.array(it1) * Ns)) / t1
    return {"workload": f"64 RVEs, sizes from {list(BATCH_SIZES)}^3, random spheres (contrast log-uniform 1e-3..1e3) "
                        "or 50-grain cubic Voronoi, 6 unit loads each (384 items), FP32 + FP64 refinement, "
                        f"tol 1e-6, budget {budget} evaluations per item",
            "size_classes": nclass, "voxel_iter_per_s_batched": vb, "voxel_iter_per_s_one_by_one": v1,
            "speedup": vb / v1, "s_batched": tb, "s_one_by_one": t1,
            "items_converged": int(np.sum(ob["item_status"] == 0)), "evaluations_total": int(np.sum(ob["iters"])),
            "same_evaluations_one_by_one": bool(np.array_equal(ob["iters"], np.array(it1))),
            "gpu_launches_batched": launches_b}


def serving_leg(hs, dev, n=40, rate=2.0, sizes=(64, 96, 128)):
    """A Poisson-arrival stream through the serving runtime: the request mix of the serving
    configuration (random spheres with contrast log-uniform in 1e-3..1e3, 5 % voids, 5 % rigid
    surrogate, or 50-grain Voronoi; 1-6 load cases) at sizes up to 128^3, FP32 + FP64 refinement,
    err <= 1e-6 or 3000 evaluations, a 150 GB budget."""
    from paper_2405_11168_gb300 import serve

    reqs = serve.synthetic_requests(n, list(sizes), 5, hs.HS_FP32_REFINED, TOL, 3000)
    srv = serve.Server(int(150 * 2 ** 30), slots=8, device=dev)
    try:
        res, wall = serve.run_stream(srv, reqs, rate, seed=5)
    finally:
        srv.close()
    solves = sum(len(r.iters) for r in res)
    return {"workload": f"{n} requests, sizes {list(sizes)}^3, Poisson arrivals at {rate} /s, 8 slots, 150 GB budget, "
                        "FP32 + FP64 refinement, tol 1e-6, budget 3000 evaluations per solve",
            "solves_per_s": solves / wall, "solves": solves, "wall_s": wall,
            "converged": sum(int(st == hs.HS_OK) for r in res for st in r.status), **serve.latency_stats(res),
            "contexts_created": srv.created, "contexts_released": srv.released, "max_running": srv.max_running,
            "max_resident_gb": srv.max_used / 2 ** 30}


def torch_stream(dev):
    import torch

    return torch.cuda.Stream(dev)


def cuda_time(dev, stream):
    """Host clock after the stream drained (the legs above are timed end to end on the host)."""
    stream.synchronize()
    import torch

    torch.cuda.synchronize(dev)
    return time.perf_counter()



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

    def solve_one(s, E, contrast=None):
        E = np.ascontiguousarray(E)
        sig_eff = np.zeros(6)
        it = ctypes.c_int()
        err = ctypes.c_double()
        st = s.lib.hs_solve(s.ctx, hs._dp(E), TOL, BUDGET, ctypes.c_void_p(eps_buf.data_ptr()),
                            ctypes.c_void_p(sig_buf.data_ptr()), hs._dp(sig_eff), ctypes.byref(it),
                            ctypes.byref(err))
        if st < 0:
            raise RuntimeError(f"solve failed: status {st}, err {err.value}")
        conv_log.append({"contrast": contrast, "status": int(st), "iters": int(it.value), "err": float(err.value)})
        return it.value, sig_eff

    def step():
        iters = 0
        C = []
        for s, c in zip(solvers, CONTRASTS):
            Ceff = np.zeros((6, 6))
            for J, E in enumerate(loads):
                k, se = solve_one(s, E, c)
                iters += k
                Ceff[:, J] = se
            C.append(Ceff)
        return iters, C

    for _ in range(args.warmup):
        step()
    for s in solvers:
        s.profile_read()
        s.profile(PROFILE_EVERY)
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
    # GB/s of the algorithmic bytes for the HBM-side kernels; the FP64 sweep is bound by the FP64
    # pipe (ncu at 128^3: 83% busy), so a bandwidth figure would not describe it
    breakdown = {k: {"ms": round(t, 3), "launches": n,
                     "ms_per_launch": round(t / n, 4) if n else None,
                     "gbs": (round(algorithmic_bytes(k, GRID) / (t / n / 1e3) / 1e9, 1)
                             if n and algorithmic_bytes(k, GRID) and k not in ("resid64", "fields") else None),
                     **({"bound": "fp64 pipe"} if k in ("resid64", "fields") else {})}
                 for k, (t, n) in prof.items() if n}

    # end to end: host ids in (pinned host memory), C_eff out, through the C ABI each step
    e2e = None
    if not args.skip_e2e:
        host_mem = "pinned"
        try:
            ids_host = torch.from_numpy(ids).pin_memory().numpy()  # hs_create copies from this buffer
        except Exception:  # noqa: BLE001 - pageable memory still gives an end-to-end number
            ids_host, host_mem = ids, "pageable"
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(args.steps):
            for t in tables:
                s = hs.Solver(ids_host, t, precision=prec, device=dev, stream=stream)
                for E in loads:
                    k, se = solve_one(s, E, None)
                    e_iters += k
                s.close()
                del s
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        e2e_ms, e_iters = combine_over_ranks(1e3 * (time.perf_counter() - t0), e_iters, dev, world)
        e2e_s = e2e_ms / 1e3
        e2e = {"value": e_iters * N / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(world * len(tables) * (ids.nbytes + 2 * 36 * 8)),
               "d2h_bytes_per_step": int(world * len(tables) * 6 * 6 * 8), "host_memory": host_mem}

    # the same iteration through torch.fft (cuFFT) and torch elementwise kernels, outside the timed region
    lib_base = None
    if rank == 0 and not args.skip_torch:
        for s in solvers:
            s.close()
        solvers = []
        torch.cuda.empty_cache()
        t_ms, t_err, fft_ms = time_torch_pipeline(ids, tables[0], dev, iters=TORCH_ITERS)
        ours_ms = sum(t / n for k, (t, n) in prof.items() if n and k in ("xpass", "y_fwd", "z_green", "y_inv",
                                                                       "x_inv", "x_fwd"))
        lib_base = {"value": N / (t_ms / 1e3), "unit": UNIT, "ms_per_iter": round(t_ms, 3),
                    "kind": "torch.fft (cuFFT) + torch elementwise ops, FP32, the same iteration",
                    "sample": f"{TORCH_ITERS} iterations of the {GRID[0]}^3 contrast-{CONTRASTS[0]:g} E11 solve "
                              f"(err after them {t_err:.3e})",
                    "cufft_transforms_ms_per_iter": round(fft_ms, 4),
                    "ours_fp32_ms_per_iter": round(ours_ms, 4),
                    "speedup_fp32_iteration": round(t_ms / ours_ms, 2) if ours_ms else None}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        one = cpu_sample(ids, tables[0], workers=cores)
        t = one()
        cpu = {"value": N / t, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "one Algorithm-1 iteration (evaluation + update) of the 256^3 contrast-1e3 E11 solve, "
                         f"{t:.1f} s"}

    legs = {}
    if rank == 0 and world == 1:
        # the oracle's own error at one timed solve's final state (contrast CONTRASTS[0], E11)
        if not args.skip_cpu:
            s0 = hs.Solver(ids_dev, tables[0], precision=prec, device=dev, stream=stream)
            o = s0.solve(loads[0], tol=TOL, max_iter=BUDGET, fields=False)
            legs["err_vs_oracle"] = dict(state_check(s0, ids, tables[0], loads[0], o["err"], o["sig_eff"]),
                                         what=f"the {GRID[0]}^3 contrast-{CONTRASTS[0]:g} E11 solve of the step "
                                              f"({BUDGET} evaluations): the oracle's FP64 evaluation (Algorithm 1 "
                                              "steps 1-4) at the GPU's final displacement")
            s0.close()
        for name, fn in (("correction_solves", lambda: correction_leg(hs, ids_dev, tables[0], dev, stream)),
                         ("converged_256", lambda: converged_256_leg(hs, ids, ids_dev, dev, stream)),
                         ("converged", lambda: converged_leg(hs, dev)),
                         ("batched", lambda: batched_leg(hs, dev)),
                         ("serving", lambda: serving_leg(hs, dev))):
            if name in args.skip_legs:
                continue
            try:
                torch.cuda.empty_cache()
                legs[name] = fn()
            except Exception as e:  # noqa: BLE001 - a leg that fails is reported, the line still prints
                legs[name] = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config("FP32 iterations + FP64 residual sweeps"),
                           parallelism=f"replicas x{world}"),
            "iterations_per_step": total_iters / args.steps,
            "solves_converged": f"{sum(x['status'] == 0 for x in timed_conv)}/{len(timed_conv)}",
            "final_err_max": max(x["err"] for x in timed_conv),
            "per_contrast": per_contrast(timed_conv),
            "roofline": roof, "kernels": breakdown,
            "kernel_timing": f"CUDA events on the solver stream: one iteration chunk in {PROFILE_EVERY} (plain "
                             "launches) and every launch outside the chunks; the other chunks replay CUDA graphs",
            "cpu_baseline": cpu, "e2e": e2e,
            "model_frac": {"bytes_per_voxel_iter": MODEL_BYTES, "frac": value * MODEL_BYTES / (peak * 1e9),
                           "what": "voxel-iter/s x the 4-pass model's bytes per FP32 voxel-iteration "
                                   "(30 x 4 B + 1 B) / measured HBM peak"},
            "torch_fft_baseline": lib_base,
            "gpu_launches": launches, "clocks": clocks,
            **legs,
        }
        print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# Bytes per FP32 voxel-iteration of the minimal 4-pass pipeline model (three
# complex half-spectrum components read and written by four passes, the state
# read and written once, a one-byte phase id): 30 x 4 + 1.
MODEL_BYTES = 121
TORCH_ITERS = 10
# Kernel times in the timed region come from CUDA events on one iteration chunk
# in PROFILE_EVERY (run as plain launches) and on every launch outside the
# chunks; the other chunks replay their CUDA graph as an untimed solve does.
# A solve here runs 8 chunks, so a period of 5 moves the timed chunk through
# every position in a solve instead of always timing the same ones.
PROFILE_EVERY = 5

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
    ap.add_argument("--skip-torch", action="store_true", help="skip the torch.fft comparison pipeline")
    ap.add_argument("--grid", type=int, default=256, help="cubic grid size (profiling runs use smaller cases)")
    ap.add_argument("--ncontrast", type=int, default=4, help="use the first k contrasts (profiling runs)")
    ap.add_argument("--skip-legs", default="", help="comma-separated legs to skip: correction_solves, converged_256, converged, "
                                                    "batched, serving")
    args = ap.parse_args()
    args.skip_legs = [x for x in args.skip_legs.split(",") if x]
    global GRID, CONTRASTS
    GRID = (args.grid,) * 3
    CONTRASTS = CONTRASTS[: max(1, min(4, args.ncontrast))]
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
