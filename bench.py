#!/usr/bin/env python
"""Benchmark of the RTLBFS time step (arXiv 2202.13449) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

One bench "step" is one pass of the whole hot path over the workload: for
the single-cavity workloads, ``inner`` consecutive explicit time steps
(fused face sweep, update, boundary conditions and the FP64 residual
reduction of every step), replayed as CUDA graphs; L2 is flushed between
bench steps.  Prints one JSON line (rank 0).

value      M cell-updates/s over all ranks, inputs resident in HBM, CUDA events
           on the library's stream around each bench step (max over ranks)
e2e        the same metric through the C ABI with host buffers: upload of the
           state, the steps, download of the state, all timed
roofline   the step kernel against the roof that binds it, the FP32 ALUs:
           algorithmic FP operations per cell-update (every face and gradient
           once, counted by the library on its own face arithmetic) x cells /
           average launch time, against SMs x 128 FP32 lanes x max SM clock
roofline_hbm  the same launches against the measured HBM copy bandwidth:
           algorithmic bytes (32 B per cell-update in FP32, 64 B in FP64)
cpu_baseline  the FP64 CPU oracle timed on this host on a bounded sample
N > 1      independent replicas, one per GPU (weak scaling): the workload has
           no data exchange between cavities.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, n or (nx, ny), phi, Ra, Pr, Ma, precision, inner steps, kind)
    "cavity512": dict(
        desc="differentially heated cavity 512x512, tanh stretching phi=2.0 (Eq. 74), "
             "Ra=1e8, Pr=0.71, Ma=0.1, FP32 bulk + FP64 reductions",
        nx=512, ny=512, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32", inner=1000,
        kind="cavity"),
    "cavity64": dict(
        desc="differentially heated cavity 64x64 uniform, Ra=1e3, Pr=0.71, Ma=0.1, FP64",
        nx=64, ny=64, phi=0.0, Ra=1e3, Pr=0.71, Ma=0.1, precision="fp64", inner=1000,
        kind="cavity"),
    "rb1024x512": dict(
        desc="Rayleigh-Benard 2:1 box 1024x512 uniform, periodic in x, Ra=1e6, Pr=0.71, "
             "Ma=0.1, FP32 bulk + FP64 reductions, seeded noise 1e-3",
        nx=1024, ny=512, phi=0.0, Ra=1e6, Pr=0.71, Ma=0.1, precision="fp32", inner=500,
        kind="rb"),
    "rb1024x512_steady": dict(
        desc="Rayleigh-Benard 2:1 box 1024x512 uniform, periodic in x, Ra=1e6, Pr=0.71, Ma=0.1, "
             "FP32 bulk + FP64 reductions, seeded noise 1e-3: time to a statistically steady "
             "Nusselt number",
        nx=1024, ny=512, phi=0.0, Ra=1e6, Pr=0.71, Ma=0.1, precision="fp32", sample_every=2000,
        window=25, onset=1.5, max_steps=2_000_000, kind="rb_steady"),
    "stability_fig4": dict(
        desc="stability map of Section 3.3, Fig. 4: differentially heated cavity 50x50 unit "
             "cells, Pr=0.71, V_c=0.1, Delta t=0.5, Ra in 1e3..1e8 x lattice spacing delta t in "
             "0.1..1.5, FP32, to max(R_u, R_T) < 1e-7 (above the FP32 state's residual floor "
             "of ~1.4e-8), divergence or 200k steps, all cases in one batch",
        grid_n=[50], grid_Ra=[1e3, 1e4, 1e5, 1e6, 1e7, 1e8],
        grid_kappa=[0.1, 0.15, 0.2, 0.3, 0.5, 0.7, 1.0, 1.5], dt=0.5, tol=1e-7,
        max_steps=200000, precision="fp32", kind="stability"),
    "stability_fig4_fp64": dict(
        desc="stability map of Section 3.3, Fig. 4 in FP64 with Eq. 65's 1e-9 (as the R12 "
             "residual): 50x50 unit cells, Pr=0.71, V_c=0.1, Delta t=0.5, Ra in 1e3..1e8 x "
             "delta t in 0.1..1.5, to convergence, divergence or 400k steps, one batch",
        grid_n=[50], grid_Ra=[1e3, 1e4, 1e5, 1e6, 1e7, 1e8],
        grid_kappa=[0.1, 0.15, 0.2, 0.3, 0.5, 0.7, 1.0, 1.5], dt=0.5, tol=1e-9,
        max_steps=400000, precision="fp64", kind="stability"),
    "stability_fig5": dict(
        desc="stability map of Section 3.3, Fig. 5: differentially heated cavity N x N unit "
             "cells, N in 10..200, delta t = 1, Pr=0.71, V_c=0.1, Delta t=0.5, Ra in 1e3..1e8, "
             "FP32, to max(R_u, R_T) < 1e-7, divergence or 200k steps, all cases in one batch",
        grid_n=[10, 20, 30, 50, 70, 100, 150, 200], grid_Ra=[1e3, 1e4, 1e5, 1e6, 1e7, 1e8],
        grid_kappa=[1.0], dt=0.5, tol=1e-7, max_steps=200000, precision="fp32",
        kind="stability"),
    "cavity8192": dict(
        desc="roofline probe: differentially heated cavity 8192x8192, tanh phi=2.0, Ra=1e8, "
             "Pr=0.71, Ma=0.1, FP32 bulk + FP64 reductions (state 1.07 GB per buffer, > L2)",
        nx=8192, ny=8192, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32", inner=10,
        kind="cavity"),
    "cavity8192_strips": dict(
        desc="one mesh over N GPUs: the 8192x8192 tanh (phi=2.0) cavity, Ra=1e8, Pr=0.71, "
             "Ma=0.1, FP32 bulk + FP64 reductions, split into N row strips (one per GPU) that "
             "exchange their two boundary rows before every step; N = 1: the whole mesh",
        nx=8192, ny=8192, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32", inner=10,
        kind="strips"),
    "cavity4096": dict(
        desc="profiling case: differentially heated cavity 4096x4096, tanh phi=2.0, Ra=1e8, "
             "Pr=0.71, Ma=0.1, FP32 bulk + FP64 reductions (state 268 MB per buffer, > L2)",
        nx=4096, ny=4096, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32", inner=20,
        kind="cavity"),
    "batch1024": dict(
        desc="1024 independent cavities, sides from {32,48,64,96,128,192,256}, tanh phi in "
             "[1.0,2.5], Ra log-uniform in [1e3,1e6], Pr=0.71, Ma=0.1, seed 1234; all advanced "
             "together, FP32 bulk + FP64 reductions",
        count=1024, seed=1234, precision="fp32", inner=50, kind="batch"),
    "serve": dict(
        desc="request trace: 10,000 square uniform cavities, Poisson arrivals at 200/s, side "
             "log-uniform 64..1024, Ra log-uniform 1e3..1e8, Pr in {0.71, 7.0}, seed 42; "
             "continuous batching, FP32 bulk + FP64 reductions",
        count=10000, seed=42, rate=200.0, precision="fp32", kind="serve"),
    "serve_steady": dict(
        desc="time to steady state in the request loop: the requests of the 10,000-request "
             "trace (seed 42, Poisson arrivals at 200/s, side log-uniform 64..1024, Ra "
             "log-uniform 1e3..1e8, Pr in {0.71, 7.0}) with side <= 128 and Ra <= 1e5, at "
             "their own arrival times (1,012 requests over 49 s), each run to max(R_u, R_T) "
             "< 1e-7 or 1e6 steps; continuous batching, FP32 bulk + FP64 reductions; the "
             "plain per-request FP64 form on converged requests for the comparison",
        count=10000, seed=42, rate=200.0, n_max=128, ra_max=1e5, max_steps=1_000_000,
        time_limit=300.0, tol=1e-7, precision="fp32", kind="serve"),
    "cavity512_accuracy": dict(
        desc="accuracy run of the 512x512 tanh cavity (Ra=1e8, Pr=0.71, Ma=0.1): the FP32 path "
             "(fixed-point state, FP64 reductions) against the FP64 path at step checkpoints "
             "1, 10, 100, 1e3, 1e4, 2e5",
        nx=512, ny=512, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32",
        checkpoints=[1, 10, 100, 1000, 10000, 200000], kind="accuracy"),
    "cavity512_tlbfs": dict(
        desc="the 512x512 tanh cavity of config 2 (Ra=1e8, Pr=0.71, Ma=0.1, FP32 bulk + FP64 "
             "reductions) with the original TLBFS face stage of Section 2.2 instead of RTLBFS",
        nx=512, ny=512, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp32", inner=1000,
        scheme=1, kind="cavity"),
    "schemes_ra1e3": dict(
        desc="RTLBFS against TLBFS (Sections 3.2 and 2.2) on the 64x64 uniform cavity at "
             "Ra=1e3, Pr=0.71, Ma=0.1, FP64, run to max(R_u, R_T) < 1e-9: Table 1's quantities "
             "and the time to the steady state for each face stage",
        n=64, Ra=1e3, Pr=0.71, Ma=0.1, tol=1e-9, max_steps=400000, kind="schemes"),
    "cubic80": dict(
        desc="3D cubic cavity of Section 4.4 / Table 6: 80x80x80 cells, tanh stretching "
             "phi=1.8 (Eq. 74) on all axes, Ra=1e6, Pr=0.71, V_c=0.1, cold -x / hot +x walls, "
             "adiabatic others, gravity along -z; D3Q19 lattice, lattice spacing kappa=0.5 times the "
             "smaller normal width; FP32 bulk + FP64 reductions",
        n=80, phi=1.8, Ra=1e6, Pr=0.71, Ma=0.1, kappa=0.5, precision="fp32", inner=500,
        kind="cubic"),
    "cubic80_fp64": dict(
        desc="3D cubic cavity of Section 4.4 / Table 6: 80x80x80 cells, tanh phi=1.8, Ra=1e6, "
             "Pr=0.71, V_c=0.1, D3Q19 lattice, FP64",
        n=80, phi=1.8, Ra=1e6, Pr=0.71, Ma=0.1, kappa=0.5, precision="fp64", inner=50,
        kind="cubic"),
    "table6": dict(
        desc="Table 6 of Section 4.4 on this GPU: the cost of a time step and of t* = V_c t / L "
             "= 1 for the RTLBFS and TLBFS face stages on the paper's mesh (80x80x80, tanh "
             "phi=1.8, Ra=1e6, Pr=0.71, V_c=0.1, lattice spacing kappa=0.5), FP64 and FP32",
        n=80, phi=1.8, Ra=1e6, Pr=0.71, Ma=0.1, kappa=0.5, precision="fp64", inner=100,
        kind="table6"),
    "cylinder450x300": dict(
        desc="mixed convection from a heated circular cylinder (Section 4.3): body-fitted O-mesh "
             "of 450 (around) x 300 (radial) cells, far field at 52.5 D, first spacing 0.003 D, "
             "D = 1; Re = 20, Gr = 100, Pr = 0.7, u_inf = 0.1 c_s along +x, buoyancy along the "
             "free stream; FP32 bulk + FP64 reductions",
        ni=450, nj=300, Re=20.0, Gr=100.0, Pr=0.7, precision="fp32", inner=200, kind="curv"),
    "cylinder3600x2400": dict(
        desc="roofline probe of the curvilinear kernel: the heated-cylinder O-mesh of Section 4.3 "
             "refined to 3600 (around) x 2400 (radial) cells (8.64 M cells, 138 MB of state per "
             "buffer, > L2), same far field, first spacing and physics; FP32",
        ni=3600, nj=2400, Re=20.0, Gr=100.0, Pr=0.7, precision="fp32", inner=20, kind="curv"),
    "cavity_tables": dict(
        desc="Tables 1-3 of Section 4.2 on this GPU: the differentially heated square cavity at "
             "Ra = 1e3 ... 1e8 on the paper's meshes (uniform 100^2, 150^2, 200^2, 250^2; "
             "300^2 and 400^2 stretched in Eq. 74's tanh form to first cells of 0.0004 L and "
             "0.0002 L), Pr = 0.71, V_c = 0.1, FP32, each from the conduction state to a steady "
             "state: max(R_u, R_T) < tol on the uniform meshes; on the stretched ones (time steps "
             "of 0.04-0.06 against 0.5, where a per-step tolerance says little) until the reported "
             "quantities change by less than window_tol over window_conv_times convective times "
             "L/V_c, or the time limit; centreline velocity maxima, streamfunction maximum, Nu_a "
             "(Eq. 69) and Nu_1/2 against the paper's RTLBFS values",
        tol=1e-7, max_steps=50_000_000, time_limit=300.0, window_conv_times=20.0,
        window_tol=2e-4, precision="fp32", kind="cavity_tables"),
    "cavity_ra1e8_fp64": dict(
        desc="Table 3's case (Ra = 1e8, 400^2 stretched to a first cell of 0.0002 L, Pr = 0.71, "
             "V_c = 0.1): windows of 20 convective times in FP32 from the conduction state, "
             "then the FP32 state continued in FP64 (exact conversion) in windows of 10, with "
             "the Table 3 quantities after every window",
        Ra=1e8, n=400, wall=0.0002, w32=11, w64=8, kind="fp64_continue"),
    "table4": dict(
        desc="Table 4 of Section 4.3 on this GPU: mean Nusselt number (Eq. 73) and separation "
             "angle on the heated cylinder at Re = 20, Pr = 0.7, Gr = 0, 100, 800, 1600, each run "
             "from the free stream to a steady state on the 450 x 300 O-mesh, FP32",
        ni=450, nj=300, Re=20.0, Pr=0.7, Grs=(0.0, 100.0, 800.0, 1600.0), precision="fp32",
        tol=1e-8, max_steps=5000000, kind="table4"),
    "cubic256": dict(
        desc="3D profiling case: cubic cavity 256x256x256, tanh phi=1.8, Ra=1e6, Pr=0.71, "
             "V_c=0.1, FP32 bulk + FP64 reductions (state 336 MB per buffer, > L2)",
        n=256, phi=1.8, Ra=1e6, Pr=0.71, Ma=0.1, kappa=0.5, precision="fp32", inner=20,
        kind="cubic"),
    "cavity512_fp64": dict(
        desc="differentially heated cavity 512x512, tanh phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, FP64",
        nx=512, ny=512, phi=2.0, Ra=1e8, Pr=0.71, Ma=0.1, precision="fp64", inner=100,
        kind="cavity"),
}
DEFAULT_WORKLOAD = "cavity512"
STEP3_SOURCES = ["paper_2202_13449_gb300/csrc/rtlbfs3d.cu",
                 "paper_2202_13449_gb300/csrc/rtlbfs3d_dev.cuh",
                 "paper_2202_13449_gb300/csrc/rtlbfs_dev.cuh"]
CURV_SOURCES = ["paper_2202_13449_gb300/csrc/rtlbfs_curv.cu",
                "paper_2202_13449_gb300/csrc/rtlbfs_dev.cuh"]
STEP_SOURCES = ["paper_2202_13449_gb300/csrc/rtlbfs_step.cu",
                "paper_2202_13449_gb300/csrc/rtlbfs_march.cu",
                "paper_2202_13449_gb300/csrc/rtlbfs_dev.cuh",
                "paper_2202_13449_gb300/csrc/rtlbfs_kernels.h",
                "paper_2202_13449_gb300/csrc/rtlbfs_tile.cuh",
                "paper_2202_13449_gb300/csrc/rtlbfs_persist.cu"]
# schedule kernel kinds of the 2D solver: short names and device kernel names
SCHED_NAMES = ["march", "tile", "persist"]
SCHED_KERNELS = ["rtlbfs::march_kernel", "rtlbfs::step_kernel", "rtlbfs::persist_kernel"]


def kernel_hash(sources=None) -> str:
    h = hashlib.sha256()
    for p in sources or STEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(workload: str, precision: str, kernel: str, sources=None):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(f"{workload}:{precision}:{kernel}")
        if e and e.get("kernel_hash") == kernel_hash(sources):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


_ALU_PEAKS = {}


def alu_peak(rs: int):
    """(peak T op/s, source) of the plain FP32 (rs = 4) or FP64 (rs = 8)
    arithmetic, measured on this device by the library's FMA-rate probe
    (independent FMA chains on every SM, CUDA-event timed; one FMA is one
    operation of the op count), best of three launches, cached per process."""
    if rs not in _ALU_PEAKS:
        from paper_2202_13449_gb300 import capi
        kind, reps = (capi.RATE_FP32, 200000) if rs == 4 else (capi.RATE_FP64, 5000)
        best = max(capi.fma_rate(kind, reps)[0] for _ in range(3))
        name = "FFMA" if rs == 4 else "DFMA"
        _ALU_PEAKS[rs] = (best / 1e12, f"measured: {name} rate of rtlbfs_fma_rate (best of 3, "
                                       f"{reps} x 8 chains per thread, every SM)")
    return _ALU_PEAKS[rs]


def rooflines(kernel: str, cells: int, per_launch_s: float, rs: int, traffic, clocks,
              scheme: int = 0):
    """(ALU roofline, HBM roofline) of the step kernel for launches of
    `cells` cell-updates taking per_launch_s each (face stage `scheme`)."""
    import torch
    from paper_2202_13449_gb300 import capi
    _, ops_cell, sfu_cell = capi.op_counts(scheme)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_alu, src = alu_peak(rs)
    unit = "T FP32 op/s" if rs == 4 else "T FP64 op/s"
    derived = sms * 128 * mhz * 1e6 / 1e12 if rs == 4 else None
    alu = ops_cell * cells / per_launch_s / 1e12
    alg_bytes = 8 * rs * cells  # read 4 fields + write 4 fields per cell
    hbm = alg_bytes / per_launch_s / 1e9
    peak, peak_kind = peaks()
    alu_line = {"bound": "alu", "achieved": round(alu, 3), "peak": round(peak_alu, 3),
                "unit": unit, "frac": round(alu / peak_alu, 4), "traffic": traffic,
                "kernel": kernel, "ops_per_cell_update": ops_cell,
                "sfu_ops_per_cell_update": sfu_cell, "peak_source": src,
                "alg_ops_per_launch": ops_cell * cells}
    if derived:
        alu_line["peak_derived"] = {"value": round(derived, 3), "frac": round(alu / derived, 4),
                                    "source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
    hbm_line = {"bound": "hbm", "achieved": round(hbm, 1), "peak": peak, "unit": "GB/s",
                "frac": round(hbm / peak, 4), "traffic": traffic, "kernel": kernel,
                "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": alg_bytes}
    return alu_line, hbm_line


def pinned(arrays):
    """Copies of numpy arrays in page-locked host memory."""
    import numpy as np
    import torch
    out = []
    for a in arrays:
        t = torch.empty(np.asarray(a).shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        out.append(t.numpy())
    return out


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"rtlbfs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_max(x: float, device="cuda") -> float:
    """Max of x over the ranks of the job (x itself in a one-process job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_sum(x: float, device="cuda") -> float:
    """Sum of x over the ranks of the job."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, rank: int, world: int):
    """This rank's share of independent work items (round robin)."""
    return list(items)[rank::world]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def setup_solver(capi, inputs, w):
    import numpy as np
    prec = capi.FP32 if w["precision"] == "fp32" else capi.FP64
    nx, ny = w["nx"], w["ny"]
    if w["kind"] == "cavity":
        xf = capi.tanh_faces(nx, float(nx), w["phi"])
        yf = capi.tanh_faces(ny, float(ny), w["phi"])
        s = capi.Solver(xf, yf, prec)
        dt = 0.5 * float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
        s.set_params(w["Ra"], w["Pr"], w["Ma"], dt)
        st = inputs.conduction_state(xf, yf)
    else:  # Rayleigh-Benard: periodic x, hot bottom, cold top; L = H
        xf = inputs.uniform_faces(nx)
        yf = inputs.uniform_faces(ny)
        s = capi.Solver(xf, yf, prec)
        s.set_bc(capi.WEST, capi.PERIODIC)
        s.set_bc(capi.EAST, capi.PERIODIC)
        s.set_bc(capi.SOUTH, capi.WALL_DIRICHLET, 1.0)
        s.set_bc(capi.NORTH, capi.WALL_DIRICHLET, 0.0)
        s.set_params_ref(w["Ra"], w["Pr"], w["Ma"], 0.5, float(ny), 1.0, 0.5)
        st = inputs.rb_state(xf, yf, amp=1e-3, seed=0)
    if w.get("scheme", 0):
        s.set_scheme(w["scheme"])
    s.set_state(*st)
    return s, st, xf, yf


def run_batch(args, w):
    """Config-4 style workload: one bench step = `inner` batched time steps of
    all cavities (one launch per step, graphs), L2 flushed between steps."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    specs = inputs.batch_specs(w["count"], w["seed"])
    prec = capi.FP32 if w["precision"] == "fp32" else capi.FP64
    b = capi.Batch(prec, len(specs))
    # a dedicated stream shared by torch (events, L2 flush) and the library;
    # the legacy default stream (handle 0) would leave the library on its own
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    b.set_stream(stream)
    cells = 0
    slots = []
    for sp in specs:
        xf = capi.tanh_faces(sp.n, float(sp.n), sp.phi)
        s = b.add(xf, xf, sp.Ra, sp.Pr, 0.1, 0.0)  # dt from the stability rule
        slots.append(s)
        cells += sp.n * sp.n
    inner = args.inner or w["inner"]
    total = inner * (args.steps + args.warmup + 64) + 1000
    for s in slots:
        b.arm(s, 0.0, total)
    if args.schedule == "auto":
        sched = b.autotune(16)
    else:
        name, _, rows = args.schedule.partition(":")
        sched = (SCHED_NAMES.index(name), int(rows or 0), 0.0)
        b.set_schedule(sched[0], sched[1])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        b.step(inner)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.step(inner)
        e.record(stream)
        ev.append((a, e))
    torch.cuda.synchronize()
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    ms = job_max(sum(a.elapsed_time(e) for a, e in ev))
    status, steps, res = b.poll()
    all_running = all(st == capi.SLOT_RUNNING for st in status[:len(specs)])
    value = cells * inner * args.steps * ws / (ms * 1e-3) / 1e6
    rs = 4 if prec == capi.FP32 else 8
    per_launch = ms * 1e-3 / (inner * args.steps)
    kname = SCHED_KERNELS[sched[0]]
    traffic = profile_traffic(args.workload, w["precision"], SCHED_NAMES[sched[0]])
    alu, hbm = rooflines(kname, cells, per_launch, rs, traffic, clocks)

    # e2e through the C ABI with host buffers: every cavity's state up from
    # pinned host memory, `inner` batched steps, every state back down
    host = {}
    for sp, s in zip(specs, slots):
        xf = capi.tanh_faces(sp.n, float(sp.n), sp.phi)
        host[s] = pinned(inputs.conduction_state(xf, xf))
    e2e_steps = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s in slots:
            b.set_state(s, *host[s])
            b.arm(s, 0.0, inner)
        b.step(inner)
        for s in slots:
            out = b.get_state(s)
    torch.cuda.synchronize()
    e2e_planes = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    # the same through the state records (rtlbfs_batch_get/set_state_raw):
    # the device's own cell records up and down, no conversion kernel
    rec_in, rec_out, tunit = {}, {}, {}
    for s in slots:
        b.set_state(s, *host[s])
        nb = b.raw_bytes(s)
        rec_in[s] = torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy()
        rec_out[s] = torch.empty(nb, dtype=torch.uint8, pin_memory=True).numpy()
        tunit[s] = b.get_state_raw(s, out=rec_in[s])[1]
    ins = [rec_in[s] for s in slots]
    outs = [rec_out[s] for s in slots]
    units = [tunit[s] for s in slots]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        b.set_states_raw(slots, ins, units)  # every slot's records in one call
        b.arm_many(slots, 0.0, inner)
        b.step(inner)
        b.get_states_raw(slots, outs)
    torch.cuda.synchronize()
    e2e = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    bytes_io = 4 * 8 * cells
    bytes_rec = 4 * rs * cells
    line = {
        "metric": "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines",
        "value": round(value, 2), "unit": "M cell-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == capi.FP32 else "f64", "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cavities": len(specs),
                   "cells": cells, "time_steps_per_bench_step": inner,
                   "state_bytes_per_buffer": 4 * rs * cells,
                   "l2": "inputs larger than L2; also flushed between bench steps",
                   "schedule": {"kernel": SCHED_NAMES[sched[0]], "chunk_rows": sched[1]},
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": round(e2e, 2), "unit": "M cell-updates/s",
                "h2d_bytes_per_step": bytes_rec, "d2h_bytes_per_step": bytes_rec,
                "api": "rtlbfs_batch_set_states_raw / rtlbfs_batch_arm_many / rtlbfs_batch_step "
                       "/ rtlbfs_batch_get_states_raw (all slots in one call each), pinned",
                "note": "per bench step: every cavity's state records uploaded from pinned host "
                        f"memory, {inner} batched time steps, every state downloaded"},
        "e2e_planes": {"value": round(e2e_planes, 2), "unit": "M cell-updates/s",
                       "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                       "api": "rtlbfs_batch_set_state / rtlbfs_batch_step / "
                              "rtlbfs_batch_get_state, pinned (four FP64 planes)"},
        "gpu_launches": int(launches),
        "roofline": alu,
        "roofline_hbm": hbm,
        "clocks": clocks,
        "all_running": all_running,
    }
    b.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch(w, args.cpu_seconds)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args, w):
    """Config-5 style workload: the request loop on a seeded trace, plus the
    plain per-request FP64 comparator on a sample of the same requests.
    With N ranks each GPU serves every N-th request of the trace (independent
    cavities: no exchange between GPUs); solves/s is the job's total over the
    slowest rank's wall time."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    trace = inputs.serving_trace(w["count"], w["seed"], w["rate"])
    # a documented sub-trace keeps the requests' own arrival times
    trace = [r for r in trace if r.n <= w.get("n_max", r.n) and r.Ra <= w.get("ra_max", r.Ra)]
    reqs = shard([(r.t_arrive, r.n, r.Ra, r.Pr) for r in trace], rank, ws)
    cap = w.get("max_steps", 2000) if args.max_steps is None else args.max_steps
    tol = w.get("tol", 1e-7) if args.tol is None else args.tol
    time_limit = w.get("time_limit", 60.0) if args.time_limit is None else args.time_limit
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    res, el = capi.serve(reqs, max_slots=args.slots, tol=tol, max_steps=cap, chunk_steps=128,
                         precision=capi.FP32, time_limit_s=time_limit, mem_fraction=0.5)
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    done = [(q, r) for q, r in zip(reqs, res) if r["status"] >= 0]
    finished_job = int(job_sum(len(done)))
    el_job = job_max(el)
    diverged = sum(1 for _, r in done if r["status"] == capi.SLOT_DIVERGED)
    retire = np.array([r["t_finish"] - q[0] for q, r in done]) if done else np.array([np.nan])
    converged = [(q, r) for q, r in done if r["status"] == capi.SLOT_CONVERGED]
    conv = len(converged)
    steady = (np.array([r["t_finish"] - q[0] for q, r in converged]) if converged
              else np.array([np.nan]))
    capped = sum(1 for _, r in done if r["status"] == capi.SLOT_MAX_STEPS)
    # plain per-request FP64 on a sample of the requests (converged ones when
    # there are any), each alone, one at a time, to the same tolerance and cap
    pool = converged if converged else done
    sample = pool[:args.fp64_sample] if rank == 0 else []
    # The accuracy of both forms against the steady state itself: each FP64
    # run is continued (untimed) to Eq. 65's 1e-9, whose mean wall Nusselt
    # number is the reference.  At a tolerance R the state still lies about
    # R x (the slowest decay time in steps) from steady, so both forms carry
    # that convergence error; the comparison is at equal tolerance.
    t64 = 0.0
    errs, errs32, errs64, conv64, steps32, steps64 = [], [], [], 0, 0, 0
    for q, r in sample:
        xf = inputs.uniform_faces(q[1])
        s = capi.Solver(xf, xf, capi.FP64)
        s.set_params(q[2], q[3], 0.1, 0.0)
        t0 = time.perf_counter()
        rc64, n64, _ = s.run_to_steady(tol, cap)
        nu64 = 0.5 * (s.nusselt(capi.NU_WEST) + s.nusselt(capi.NU_EAST))
        t64 += time.perf_counter() - t0
        conv64 += rc64 == capi.OK
        steps32 += r["steps"]
        steps64 += n64
        nu32 = 0.5 * (r["nu_hot"] + r["nu_cold"])
        errs.append(abs(nu32 - nu64) / abs(nu64))
        rc_ref = capi.ERR_NOT_CONVERGED
        if converged:  # requests stopped at a step cap are not near any steady state
            rc_ref, _, _ = s.run_to_steady(1e-9, 20 * cap)
        if rc_ref == capi.OK:
            nu_ref = 0.5 * (s.nusselt(capi.NU_WEST) + s.nusselt(capi.NU_EAST))
            errs32.append(abs(nu32 - nu_ref) / abs(nu_ref))
            errs64.append(abs(nu64 - nu_ref) / abs(nu_ref))
        s.close()
    admitted = [(q, r) for q, r in zip(reqs, res) if r["t_admit"] >= 0]
    h2d = sum(32 * q[1] * q[1] + 16 * (q[1] + 1) for q, _ in admitted)
    updates = sum(q[1] * q[1] * r["steps"] for q, r in done)
    line = {
        "metric": "batched solves/s and p50/p99 time-to-steady (request loop)",
        "value": round(finished_job / el_job, 3) if el_job > 0 else None, "unit": "solves/s",
        "n_gpus": ws, "steps": 1, "warmup": 0, "ms_per_step": round(el_job * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"],
                   "requests": len(trace), "requests_this_rank": len(reqs),
                   "max_steps_cap": cap, "tol": tol, "time_limit_s": time_limit,
                   "slots": args.slots, "parallelism": f"trace sharded over {ws} GPU(s)"},
        "finished": finished_job, "converged": conv, "hit_step_cap": capped, "diverged": diverged,
        "unfinished": len(reqs) - len(done),
        "counts_scope": "finished: the whole job; converged/capped/diverged/unfinished and the "
                        "latency percentiles: rank 0's share of the trace",
        "arrival_to_retirement_s": {"p50": float(np.nanpercentile(retire, 50)),
                                    "p99": float(np.nanpercentile(retire, 99)),
                                    "note": "every finished request (converged, capped or "
                                            "diverged)"},
        "time_to_steady_s": ({"p50": float(np.nanpercentile(steady, 50)),
                              "p99": float(np.nanpercentile(steady, 99)),
                              "requests": conv,
                              "note": "arrival to retirement of the converged requests"}
                             if conv else None),
        "fp64_per_request": {"requests": len(sample), "of": "converged" if converged else "finished",
                             "solves_per_s": round(len(sample) / t64, 3) if t64 > 0 else None,
                             "converged": conv64, "steps_fp32": steps32, "steps_fp64": steps64,
                             "max_rel_err_mean_wall_nu_fp32_vs_fp64": max(errs) if errs else None,
                             "reference": "the same FP64 run continued to max(R_u, R_T) < 1e-9",
                             "references": len(errs32),
                             "max_rel_err_mean_wall_nu_fp32_vs_reference":
                                 max(errs32) if errs32 else None,
                             "max_rel_err_mean_wall_nu_fp64_vs_reference":
                                 max(errs64) if errs64 else None},
        "e2e": {"value": round(finished_job / el_job, 3) if el_job > 0 else None,
                "unit": "solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * len(done),
                "note": "the request loop is the public call: requests from the host, "
                        "conduction states and faces uploaded per admission, Nusselt numbers "
                        "read back per retirement; one bench step = the whole trace"},
        "cell_updates_per_s_M": round(updates / el / 1e6, 1) if el > 0 else None,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        steps_by_req = [r["steps"] if r["status"] >= 0 else cap for r in res]
        line["cpu_baseline"] = cpu_baseline_serve(w, reqs, steps_by_req, args.cpu_seconds)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_accuracy(args, w):
    """FP32 against FP64 (the GPU FP64 path is tied to the oracle, step by
    step, by the parity tests) on the config-2 cavity at step checkpoints:
    field errors relative to max(max|FP64|, floor) and the mean wall Nusselt
    number's relative error."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    xf = capi.tanh_faces(w["nx"], float(w["nx"]), w["phi"])
    dt = 0.5 * float(np.min(np.diff(xf)))
    sol = {}
    for prec in (capi.FP64, capi.FP32):
        s = capi.Solver(xf, xf, prec)
        s.set_params(w["Ra"], w["Pr"], w["Ma"], dt)
        s.set_state(*inputs.conduction_state(xf, xf))
        sol[prec] = s
    rows, done, t0 = [], 0, time.perf_counter()
    worst = 0.0
    for cp in w["checkpoints"]:
        for s in sol.values():
            s.step(cp - done)
        done = cp
        a, b = sol[capi.FP32].get_state(), sol[capi.FP64].get_state()
        nu = {p: 0.5 * (sol[p].nusselt(capi.NU_WEST) + sol[p].nusselt(capi.NU_EAST)) for p in sol}
        def rel(x, y, floor):
            return float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), floor))
        row = {"step": cp, "rel_err_u": rel(a[1], b[1], 0.1), "rel_err_v": rel(a[2], b[2], 0.1),
               "rel_err_T": rel(a[3], b[3], 1.0), "abs_err_rho": float(np.max(np.abs(a[0] - b[0]))),
               "mean_wall_nu_fp64": nu[capi.FP64], "mean_wall_nu_fp32": nu[capi.FP32],
               "rel_err_nu": abs(nu[capi.FP32] - nu[capi.FP64]) / abs(nu[capi.FP64])}
        worst = max(worst, row["rel_err_u"], row["rel_err_v"], row["rel_err_T"])
        rows.append(row)
    el = time.perf_counter() - t0
    for s in sol.values():
        s.close()
    line = {"metric": "FP32 vs FP64 relative field error (max over u, v, T and checkpoints)",
            "value": worst, "unit": "relative error", "n_gpus": 1, "steps": len(rows),
            "warmup": 0, "ms_per_step": round(el * 1e3 / max(done, 1), 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (conduction initial state)",
            "config": {"workload": args.workload, "description": w["desc"],
                       "cells": w["nx"] * w["ny"], "dt": dt,
                       "norm": "max|FP32 - FP64| / max(max|FP64|, floor); floors u, v 0.1 "
                               "(V_c), T 1 (dT)"},
            "checkpoints": rows,
            "targets": {"fields": 1e-5, "mean_wall_nu": 1e-4}}
    print(json.dumps(line), flush=True)


def run_rb_steady(args, w):
    """Config 3's second figure: from the seeded initial state, step until
    the wall Nusselt numbers are statistically steady and report the steps
    and device time it took.  Steady: convection has set in (a wall value
    above `onset`; the perturbation grows from 1e-3, so Nu first sits at its
    conduction value 1 for many free-fall times), and over the last `window`
    samples (one every `sample_every` steps) the bottom and top means agree
    within 5 % and their mean moved less than 2 % against the window before."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    s, _, _, _ = setup_solver(capi, inputs, dict(w, kind="rb"))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream)
    sched = s.autotune(32)  # on a snapshot of the initial state, restored
    k, W = w["sample_every"], w["window"]
    # the library's wall Nusselt number is the wall's heat flux / (chi dT);
    # per unit wall length and across the layer height that is x (H / width)
    aspect = float(w["ny"]) / float(w["nx"])
    bottom, top, steps, t_dev = [], [], 0, 0.0
    steady_at, onset_at = None, None
    while steps < w["max_steps"]:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(k)
        b.record(stream)
        b.synchronize()
        t_dev += a.elapsed_time(b) * 1e-3
        steps += k
        bottom.append(s.nusselt(capi.NU_SOUTH) * aspect)
        top.append(s.nusselt(capi.NU_NORTH) * aspect)
        if onset_at is None and max(bottom[-1], top[-1]) > w["onset"]:
            onset_at = len(bottom)
        if onset_at is not None and len(bottom) - onset_at >= 2 * W:
            m_now = 0.5 * (np.mean(bottom[-W:]) + np.mean(top[-W:]))
            m_prev = 0.5 * (np.mean(bottom[-2 * W:-W]) + np.mean(top[-2 * W:-W]))
            gap = abs(np.mean(bottom[-W:]) - np.mean(top[-W:])) / abs(m_now)
            if gap < 0.05 and abs(m_now - m_prev) / abs(m_now) < 0.02:
                steady_at = steps
                break
    cells = w["nx"] * w["ny"]
    res, _ = s.residual()
    s.close()
    m = 0.5 * (np.mean(bottom[-W:]) + np.mean(top[-W:]))
    line = {"metric": "time to a statistically steady Nusselt number (device time)",
            "value": round(t_dev, 3) if steady_at else None, "unit": "s",
            "n_gpus": 1, "steps": steps, "warmup": 0,
            "ms_per_step": round(t_dev * 1e3 / max(steps, 1), 5), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded noise, seed 0)",
            "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                       "criterion": f"after the onset of convection (a wall Nu > {w['onset']}), over "
                                    f"the last {W} samples (every {k} steps) bottom and top mean "
                                    "Nu within 5 % and the mean moved < 2 % against the previous "
                                    "window; Nu per unit wall length across the layer height"},
            "schedule": {"kernel": SCHED_NAMES[sched[0]], "chunk_rows": sched[1]},
            "steady_at_step": steady_at, "onset_at_step": onset_at * k if onset_at else None,
            "nusselt_mean": m,
            "nusselt_bottom_last": bottom[-1], "nusselt_top_last": top[-1],
            "throughput_M_cell_updates_per_s": round(cells * steps / t_dev / 1e6, 1),
            "residual_last_step": res,
            "nu_history_every_k": {"bottom": [round(x, 5) for x in bottom],
                                   "top": [round(x, 5) for x in top]}}
    print(json.dumps(line), flush=True)


def stability_cases(w):
    return [(n, Ra, k) for n in w["grid_n"] for Ra in w["grid_Ra"] for k in w["grid_kappa"]]


def run_stability(args, w):
    """Section 3.3's stability maps through rtlbfs_stability_map: every
    (N, Ra, delta t) case of the grid in one batch, each run until it
    converges, diverges or hits the step cap."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2202_13449_gb300 import capi
    capi.lib()
    cases = stability_cases(w)
    n, Ra, kappa = (np.array(c) for c in zip(*cases))
    prec = capi.FP32 if w["precision"] == "fp32" else capi.FP64
    clk = ClockSampler(0)
    clk.start()
    l0 = capi.launch_count()
    status, steps, el = capi.stability_map(n, Ra, kappa, np.full(len(cases), w["dt"]),
                                           tol=w["tol"], max_steps=w["max_steps"],
                                           precision=prec, chunk_steps=256)
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    name = {capi.SLOT_CONVERGED: "converged", capi.SLOT_DIVERGED: "diverged",
            capi.SLOT_MAX_STEPS: "step cap"}
    updates = float(np.sum(steps * n.astype(np.float64) ** 2))
    # Fig. 4's trend: at each (N, Ra) the cases that did not diverge form an
    # upper range of delta t
    trend = True
    for nn in w["grid_n"]:
        for ra in w["grid_Ra"]:
            row = [status[k] for k, c in enumerate(cases) if c[0] == nn and c[1] == ra]
            ok = [x != capi.SLOT_DIVERGED for x in row]
            trend = trend and all(ok[i] <= ok[i + 1] for i in range(len(ok) - 1))
    line = {"metric": "stability map: M cell-updates/s of the batched cases (wall time of the "
                      "call)",
            "value": round(updates / el / 1e6, 2) if el > 0 else None,
            "unit": "M cell-updates/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": round(el * 1e3, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": w["precision"].replace("fp", "f"),
            "data": "synthetic (conduction initial state)",
            "config": {"workload": args.workload, "description": w["desc"], "cases": len(cases)},
            "e2e": {"value": round(updates / el / 1e6, 2) if el > 0 else None,
                    "unit": "M cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0,
                    "note": "the call is the public API: cases in, outcomes out; states are "
                            "built on the device"},
            "gpu_launches": int(launches), "clocks": clocks,
            "wall_s": round(el, 3),
            "map": [{"N": int(c[0]), "Ra": c[1], "delta_t": c[2], "outcome": name.get(int(st)),
                     "steps": int(sp)} for c, st, sp in zip(cases, status, steps)],
            "counts": {v: int(np.sum(status == k)) for k, v in name.items()},
            "small_delta_t_diverges_trend": trend}
    print(json.dumps(line), flush=True)


# Table 1 of the paper at Ra = 1e3: the RTLBFS ("Present") and TLBFS [24] rows
TABLE1_RA1E3 = {
    "rtlbfs": {"u_max": 3.644, "y_u": 0.814, "v_max": 3.698, "x_v": 0.180, "Nu_a": 1.118},
    "tlbfs": {"u_max": 3.640, "y_u": 0.815, "v_max": 3.708, "x_v": 0.180, "Nu_a": 1.115},
}


def run_schemes(args, w):
    """Both face stages to the steady state of the Ra = 1e3 cavity on the
    GPU in FP64: Table 1's quantities and the device time each needs."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    n = w["n"]
    xf = inputs.uniform_faces(n)
    out = {}
    for name, scheme in (("rtlbfs", capi.RTLBFS), ("tlbfs", capi.TLBFS)):
        s = capi.Solver(xf, xf, capi.FP64)
        s.set_params(w["Ra"], w["Pr"], w["Ma"], 0.5)
        s.set_scheme(scheme)
        s.set_state(*inputs.conduction_state(xf, xf))
        s.autotune(16)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, steps, res = s.run_to_steady(w["tol"], w["max_steps"])
        el = time.perf_counter() - t0
        st = s.get_state()
        nu_a = s.nusselt(capi.NU_AVG)
        nu_w = 0.5 * (s.nusselt(capi.NU_WEST) + s.nusselt(capi.NU_EAST))
        s.close()
        nu, chi = 0.1 * n * np.sqrt(w["Pr"] / w["Ra"]), 0.1 * n * np.sqrt(w["Pr"] / w["Ra"]) / w["Pr"]
        u_c = 0.5 * (st[1][:, n // 2 - 1] + st[1][:, n // 2])
        v_c = 0.5 * (st[2][n // 2 - 1, :] + st[2][n // 2, :])
        yc = (np.arange(n) + 0.5) / n
        out[name] = {"converged": rc == 0, "steps": int(steps), "wall_s": round(el, 3),
                     "ms_per_step": round(el * 1e3 / max(steps, 1), 4),
                     "u_max": float(u_c.max() * n / chi), "y_u": float(yc[u_c.argmax()]),
                     "v_max": float(v_c.max() * n / chi), "x_v": float(yc[v_c.argmax()]),
                     "Nu_a": float(nu_a), "Nu_wall_mean": float(nu_w),
                     "paper_table1": TABLE1_RA1E3[name]}
    ratio = out["tlbfs"]["ms_per_step"] / out["rtlbfs"]["ms_per_step"]
    line = {"metric": "time per step of TLBFS over RTLBFS (FP64, 64x64, to the steady state)",
            "value": round(ratio, 3), "unit": "ratio", "n_gpus": 1, "steps": 2, "warmup": 0,
            "ms_per_step": out["rtlbfs"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (conduction initial state)",
            "config": {"workload": args.workload, "description": w["desc"]},
            "schemes": out,
            "note": "the paper's Table 6 compares the two solvers' cost in 3D; here the face "
                    "stages share mesh, update and reductions"}
    print(json.dumps(line), flush=True)


def cubic_setup(capi, inputs, w):
    """The 3D cubic cavity of a workload: solver, initial state, faces."""
    n = w["n"]
    f = capi.tanh_faces(n, float(n), w["phi"])
    prec = capi.FP32 if w["precision"] == "fp32" else capi.FP64
    s = capi.Solver3(f, f, f, prec)
    dt = 0.5 * float(min(f[1:] - f[:-1]))
    s.set_params(w["Ra"], w["Pr"], w["Ma"], dt)
    s.set_lattice(w.get("kappa", 1.0))
    st = inputs.conduction_state3(f, f, f)
    s.set_state(*st)
    return s, st, f, dt


def run_cubic(args, w):
    """3D workload: one bench step = `inner` time steps of the cubic cavity
    (one launch per step, graphs), L2 flushed between bench steps."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    n = w["n"]
    cells = n ** 3
    inner = args.inner or w["inner"]
    s, st0, f, dt = cubic_setup(capi, inputs, w)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream)
    if args.schedule == "auto":
        tile, tune_ms = s.autotune(max(8, min(64, 20_000_000 // cells + 8)))
    else:
        tile = int(args.schedule.split(":")[1]) if ":" in args.schedule else 0
        s.set_schedule(tile, 0)
        tune_ms = 0.0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        s.step(inner)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    ev = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(inner)
        b.record(stream)
        ev.append((a, b))
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    ms_max = job_max(sum(a.elapsed_time(b) for a, b in ev))
    value = cells * inner * args.steps * ws / (ms_max * 1e-3) / 1e6

    host = pinned(st0)
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(*host)
        s.step(inner)
        out = s.get_state()
    torch.cuda.synchronize()
    e2e = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    assert np.all(np.isfinite(out[4]))
    bytes_io = 5 * cells * 8

    per_launch_s = ms_max * 1e-3 / (inner * args.steps)
    rs = 4 if w["precision"] == "fp32" else 8
    _, ops_cell, sfu_cell = capi.op_counts3()
    peak_alu, src = alu_peak(rs)
    unit = "T FP32 op/s" if rs == 4 else "T FP64 op/s"
    traffic = profile_traffic(args.workload, w["precision"], "step3", STEP3_SOURCES)
    alu = ops_cell * cells / per_launch_s / 1e12
    alg_bytes = 10 * rs * cells  # read 5 fields + write 5 fields per cell
    hbm = alg_bytes / per_launch_s / 1e9
    peak, peak_kind = peaks()
    # Table 6 context: device time for t* = V_c t / L = 1 on this mesh
    steps_t1 = int(np.ceil(float(n) / (w["Ma"] * dt)))
    res, steps_total = s.residual()
    line = {
        "metric": "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines",
        "value": round(value, 2),
        "unit": "M cell-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if rs == 4 else "f64",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "time_steps_per_bench_step": inner, "parallelism": f"replicas x{ws}",
                   "l2": "flushed between bench steps (256 MB write)",
                   "schedule": {"kernel": "step3", "tile": ["32x4", "16x8", "32x8"][tile],
                                "autotune_ms_per_step": round(tune_ms, 5)},
                   "dt": dt, "e2e_host_buffers": "pinned",
                   "state_bytes_per_buffer": 5 * rs * cells},
        "e2e": {"value": round(e2e, 2), "unit": "M cell-updates/s",
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": round(alu, 3), "peak": round(peak_alu, 3),
                     "unit": unit, "frac": round(alu / peak_alu, 4), "traffic": traffic,
                     "kernel": "rtlbfs3::step3_kernel", "ops_per_cell_update": ops_cell,
                     "sfu_ops_per_cell_update": sfu_cell, "peak_source": src,
                     "alg_ops_per_launch": ops_cell * cells},
        "roofline_hbm": {"bound": "hbm", "achieved": round(hbm, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(hbm / peak, 4), "traffic": traffic,
                         "kernel": "rtlbfs3::step3_kernel",
                         "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": alg_bytes},
        "table6_context": {"steps_for_t_star_1": steps_t1,
                           "device_s_for_t_star_1": round(steps_t1 * per_launch_s, 3),
                           "paper_rtlbfs_s": 58864.12, "paper_tlbfs_s": 60585.58,
                           "paper_hardware": "serial CPU program, machine unspecified"}
        if n == 80 else None,
        "clocks": clocks,
        "wall_s": round(t_wall, 3),
        "residual_last_step": res,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_cubic(w, args.cpu_seconds)
    if ws > 1:
        torch.distributed.destroy_process_group()
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_cubic(w):
    import oracle
    from oracle import d3
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    n = w["n"]
    f = oracle.tanh_faces(n, float(n), w["phi"])
    p = d3.cubic_cavity(n, w["Ra"], Pr=w["Pr"], Ma=w["Ma"], phi=w["phi"], kappa=w.get("kappa", 1.0))
    st = inputs.conduction_state3(f, f, f)
    return oracle, d3, p, st


def cpu_baseline_cubic(w, seconds):
    """The 3D FP64 oracle as it stands on this host's cores: time steps of the
    same mesh until `seconds` (at least one)."""
    oracle, d3, p, st = oracle_cubic(w)
    used = oracle.set_threads(os.cpu_count() or 1)
    cells = w["n"] ** 3
    n, t0 = 0, time.perf_counter()
    while n == 0 or time.perf_counter() - t0 < seconds:
        st, _, _ = d3.step(p, st, 1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": round(cells * n / dt / 1e6, 3), "unit": "M cell-updates/s", "cores": used,
            "kind": "oracle",
            "sample": f"{n} FP64 time steps of the same {w['n']}^3 mesh ({dt:.1f} s, OpenMP "
                      f"over z-planes)"}


def run_table6(args, w):
    """Per-step device time of both face stages on the Table 6 mesh, each
    precision; the line's value is the RTLBFS / TLBFS cost ratio in FP64 (the
    paper's 97.16 % was for serial CPU programs)."""
    import numpy as np
    import torch
    from paper_2202_13449_gb300 import capi, inputs
    torch.cuda.set_device(0)
    capi.lib()
    n = w["n"]
    cells = n ** 3
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    launches0 = capi.launch_count()
    clk = ClockSampler(0)
    clk.start()
    for prec_name, prec, inner in (("fp64", capi.FP64, max(20, args.inner or 50)),
                                   ("fp32", capi.FP32, max(100, (args.inner or 50) * 10))):
        for scheme, sname in ((0, "rtlbfs"), (1, "tlbfs")):
            ww = dict(w, precision=prec_name)
            s, st0, f, dt = cubic_setup(capi, inputs, ww)
            s.set_scheme(scheme)
            s.set_stream(stream)
            tile, _ = s.autotune(8)
            for _ in range(args.warmup):
                s.step(inner)
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(inner)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b) / inner)
            per = statistics.median(ms)
            steps_t1 = int(np.ceil(float(n) / (w["Ma"] * dt)))
            out[f"{sname}_{prec_name}"] = {
                "ms_per_step": round(per, 5), "M_cell_updates_per_s": round(cells / per / 1e3, 2),
                "t_cost_s_for_t_star_1": round(per * steps_t1 / 1e3, 3),
                "tile": ["32x4", "16x8", "32x8"][tile],
                "ops_per_cell_update": capi.op_counts3(scheme)[1]}
            s.close()
    clocks = clk.stop()
    ratio64 = out["rtlbfs_fp64"]["ms_per_step"] / out["tlbfs_fp64"]["ms_per_step"]
    ratio32 = out["rtlbfs_fp32"]["ms_per_step"] / out["tlbfs_fp32"]["ms_per_step"]
    line = {
        "metric": "RTLBFS / TLBFS cost ratio per time step (Table 6's t_cost ratio), FP64",
        "value": round(ratio64, 4), "unit": "ratio", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "l2": "state in L2 (20 MB FP64); median of per-bench-step timings"},
        "fp32_ratio": round(ratio32, 4),
        "stages": out,
        "paper": {"rtlbfs_s": 58864.12, "tlbfs_s": 60585.58, "ratio": 0.9716,
                  "hardware": "serial CPU programs, machine unspecified"},
        "gpu_launches": int(capi.launch_count() - launches0),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_table4(args, w):
    """Table 4 on the GPU: each Gr case from the free stream to a steady state
    (max(R_u, R_T) < tol, checked on the device every step), then Eq. 73's
    mean Nusselt number and the separation angles from the state.  The
    line's value is the largest relative deviation of Nu from the paper's
    RTLBFS column."""
    import torch
    from paper_2202_13449_gb300 import capi, inputs, post
    torch.cuda.set_device(0)
    capi.lib()
    with open(os.path.join(ROOT, "tests", "golden", "table4_cylinder.json")) as f:
        gold = {c["Gr"]: c for c in json.load(f)["cases"]}
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    launches0 = capi.launch_count()
    clk = ClockSampler(0)
    clk.start()
    rows, worst, total_ms, total_steps = [], 0.0, 0.0, 0
    for Gr in w["Grs"]:
        s, st0, XY, phys = curv_setup(capi, inputs, dict(w, Gr=Gr))
        s.set_stream(stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc, steps, res = s.run_to_steady(w["tol"], w["max_steps"], timeout_s=600.0)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        heat, perim = s.wall_heat(2)
        nu_cyl = heat / (phys["chi"] * perim)  # Eq. 73 with D = dT = 1
        rho, u, v, T = s.get_state()
        th = post.separation_angle(XY[0], XY[1], u, v)
        g = gold[Gr]
        dev = abs(nu_cyl - g["Nu"]) / g["Nu"]
        worst = max(worst, dev)
        total_ms += ms
        total_steps += steps
        rows.append({"Gr": Gr, "status": rc, "steps": steps, "residual": res,
                     "Nu": round(nu_cyl, 4), "Nu_paper": g["Nu"], "Nu_rel_dev": round(dev, 4),
                     "theta_s_deg": [round(t, 2) for t in th], "theta_s_paper": g["theta_s_deg"],
                     "device_s": round(ms / 1e3, 2)})
        s.close()
    clocks = clk.stop()
    cells = w["ni"] * w["nj"]
    line = {
        "metric": "max relative deviation of the mean cylinder Nusselt number from Table 4",
        "value": round(worst, 4), "unit": "ratio", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "tol": w["tol"], "dt": phys["dt"]},
        "cases": rows,
        "throughput_M_cell_updates_per_s": round(cells * total_steps / (total_ms * 1e-3) / 1e6, 1),
        "gpu_launches": int(capi.launch_count() - launches0),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def stretch_to_first_cell(n, L, w1):
    """The phi of Eq. 74's tanh faces on [0, L] whose first cell is w1 wide
    (the first width falls as phi grows; bisection)."""
    from paper_2202_13449_gb300 import capi
    lo, hi = 1e-3, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = capi.tanh_faces(n, L, mid)
        if f[1] - f[0] > w1:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def run_cavity_tables(args, w):
    """Tables 1-3 on the GPU: each case from the conduction state to a
    steady state (max(R_u, R_T) < tol, the step cap or the time limit),
    then the paper's quantities from the state and the Nusselt reductions.
    The line's value is the largest relative deviation of the velocity,
    streamfunction and Nusselt maxima of the converged cases from the
    paper's RTLBFS values."""
    import numpy as np
    import torch
    from paper_2202_13449_gb300 import capi, inputs, post
    torch.cuda.set_device(0)
    capi.lib()
    with open(os.path.join(ROOT, "tests", "golden", "tables123_cavity.json")) as f:
        gold = json.load(f)
    Pr, Vc = gold["Pr"], gold["Vc"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    launches0 = capi.launch_count()
    clk = ClockSampler(0)
    clk.start()
    max_steps = args.max_steps or w["max_steps"]
    tlim = args.time_limit or w["time_limit"]
    tol = args.tol or w["tol"]
    rows, worst, cu, total_ms = [], 0.0, 0.0, 0.0
    for g in gold["cases"]:
        n, L = g["n"], float(g["n"])
        if g["wall"] > 0.0:
            phi = stretch_to_first_cell(n, L, g["wall"] * L)
            xf = capi.tanh_faces(n, L, phi)
        else:
            phi = 0.0
            xf = inputs.uniform_faces(n, L)
        s = capi.Solver(xf, xf, capi.FP32)
        s.set_params(g["Ra"], Pr, Vc, 0.0)  # dt by the library's stability rule
        s.set_stream(stream)
        s.autotune(32)  # this mesh's schedule, on a snapshot of the initial state
        nu = Vc * L * np.sqrt(Pr / g["Ra"])  # the library's mapping (Eq. 63, V_c = Ma)
        chi = nu / Pr
        wmin = float(np.min(np.diff(xf)))
        dt = min(0.5 * wmin, 0.2 * wmin * wmin / max(nu, chi))  # the library's rule

        def quantities():
            rho, u, v, T = s.get_state()
            umax, uy, vmax, vx = post.cavity_centrelines(xf, xf, u, v)
            q = {"u_max": umax * L / chi, "u_max_y": uy, "v_max": vmax * L / chi,
                 "v_max_x": vx, "Nu_a": s.nusselt(capi.NU_AVG),
                 "Nu_half": s.nusselt(capi.NU_HALF)}
            pmax, px, py = post.streamfunction_max(xf, xf, u)
            q.update({"psi_max": pmax / chi, "psi_max_x": px, "psi_max_y": py})
            return q

        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        windows, change = 0, None
        if g["wall"] == 0.0:
            a.record(stream)
            rc, steps, res = s.run_to_steady(tol, max_steps, timeout_s=tlim)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            got = quantities()
        else:
            chunk = int(round(w["window_conv_times"] * (L / Vc) / dt))
            t0 = time.time()
            steps, ms, prev, rc, got = 0, 0.0, None, capi.ERR_TIMEOUT, None
            while time.time() - t0 < tlim and steps + chunk <= max_steps:
                a.record(stream)
                s.step(chunk)
                b.record(stream)
                b.synchronize()
                ms += a.elapsed_time(b)
                steps += chunk
                windows += 1
                got = quantities()
                keys = ("u_max", "v_max", "Nu_a", "Nu_half", "psi_max")
                if prev is not None:
                    change = max(abs(got[k] - prev[k]) / abs(got[k]) for k in keys)
                    if change < w["window_tol"]:
                        rc = 0
                        break
                prev = got
            if got is None:  # no window fitted in the limits
                got = quantities()
            (res_u, res_T), _ = s.residual()
            res = [res_u, res_T]
        total_ms += ms
        cu += float(n * n) * steps
        s.close()
        dev = {}
        for k, ref in g.items():
            if k in ("Ra", "n", "wall"):
                continue
            if k.endswith(("_x", "_y")):
                dev[k] = round(abs(got[k] - ref), 4)  # positions: absolute, in L
            else:
                dev[k] = round(abs(got[k] - ref) / abs(ref), 4)
                if rc == 0:
                    worst = max(worst, dev[k])
        rows.append({"Ra": g["Ra"], "n": n, "phi": round(phi, 5), "status": rc, "steps": steps,
                     "dt": dt, "residual": res, "device_s": round(ms / 1e3, 2),
                     "windows": windows, "last_window_change": change,
                     "got": {k: round(v2, 5) for k, v2 in got.items()},
                     "paper": {k: g[k] for k in dev}, "deviation": dev})
    clocks = clk.stop()
    line = {
        "metric": "max relative deviation from the paper's Tables 1-3 (converged cases)",
        "value": round(worst, 4), "unit": "ratio", "n_gpus": 1, "steps": 1, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "tol": tol,
                   "max_steps": max_steps, "time_limit_s": tlim},
        "cases": rows,
        "throughput_M_cell_updates_per_s": round(cu / (total_ms * 1e-3) / 1e6, 1),
        "gpu_launches": int(capi.launch_count() - launches0),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_fp64_continue(args, w):
    """One cavity case in FP32 windows (20 convective times each), then its
    state continued in FP64 (windows of 10): whether a quantity the FP32
    state has stopped moving is at its steady value, or frozen by the
    fixed-point quantum at a small time step."""
    import numpy as np
    import torch
    from paper_2202_13449_gb300 import capi, post
    torch.cuda.set_device(0)
    capi.lib()
    Pr, Vc = 0.71, 0.1
    n, L = w["n"], float(w["n"])
    xf = capi.tanh_faces(n, L, stretch_to_first_cell(n, L, w["wall"] * L))
    nu = Vc * L * np.sqrt(Pr / w["Ra"])
    chi = nu / Pr
    wmin = float(np.min(np.diff(xf)))
    dt = min(0.5 * wmin, 0.2 * wmin * wmin / max(nu, chi))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def quantities(s):
        rho, u, v, T = s.get_state()
        umax, uy, vmax, vx = post.cavity_centrelines(xf, xf, u, v)
        pmax, px, py = post.streamfunction_max(xf, xf, u)
        return {"u_max": round(umax * L / chi, 4), "u_max_y": round(uy, 5),
                "v_max": round(vmax * L / chi, 3), "Nu_half": round(s.nusselt(capi.NU_HALF), 5),
                "psi_max": round(pmax / chi, 5)}

    windows = {"fp32": [], "fp64": []}
    chunk = int(round(20.0 * (L / Vc) / dt))
    s = capi.Solver(xf, xf, capi.FP32)
    s.set_params(w["Ra"], Pr, Vc, 0.0)
    s.set_stream(stream)
    s.autotune(32)
    for _ in range(w["w32"]):
        s.step(chunk)
        windows["fp32"].append(quantities(s))
    st = s.get_state()
    s.close()
    d = capi.Solver(xf, xf, capi.FP64)
    d.set_params(w["Ra"], Pr, Vc, 0.0)
    d.set_stream(stream)
    d.set_state(*st)
    d.autotune(4)
    for _ in range(w["w64"]):
        d.step(chunk // 2)
        windows["fp64"].append(quantities(d))
    d.close()
    print(json.dumps({"metric": "Table 3 quantities after FP32 and FP64 windows", "value": None,
                      "unit": None, "n_gpus": 1, "dtype": "f32 then f64",
                      "data": "synthetic (seeded; no dataset)",
                      "config": {"workload": args.workload, "description": w["desc"], "dt": dt,
                                 "steps_per_fp32_window": chunk,
                                 "steps_per_fp64_window": chunk // 2},
                      "windows": windows}), flush=True)


def curv_case(inputs, w):
    """The Section 4.3 cylinder: mesh, physics and the free-stream state."""
    import numpy as np
    X, Y = inputs.cylinder_o_mesh(w["ni"], w["nj"])
    uinf = 0.1 / np.sqrt(3.0)
    nu = uinf * 1.0 / w["Re"]
    chi = nu / w["Pr"]
    beta_g = w["Gr"] * nu * nu  # Gr = beta g dT D^3 / nu^2 with D = dT = 1
    # the smallest cell width, radial or around
    wmin = min(float(np.min(np.diff(np.hypot(X, Y), axis=0))),
               float(np.min(np.hypot(np.diff(X, axis=1), np.diff(Y, axis=1)))))
    # half the smallest width, capped by the explicit diffusive limit there
    dt = min(0.5 * wmin, 0.2 * wmin * wmin / max(nu, chi))
    nj, ni = X.shape[0] - 1, X.shape[1] - 1
    st = (np.ones((nj, ni)), np.full((nj, ni), uinf), np.zeros((nj, ni)), np.zeros((nj, ni)))
    return X, Y, st, dict(nu=nu, chi=chi, beta_g=beta_g, dt=dt, uinf=uinf)


def curv_setup(capi, inputs, w):
    """The Section 4.3 cylinder on the GPU: solver and free-stream initial state."""
    X, Y, st, phys = curv_case(inputs, w)
    prec = capi.FP32 if w["precision"] == "fp32" else capi.FP64
    s = capi.SolverC(X, Y, True, prec)
    s.set_physics(phys["nu"], phys["chi"], phys["beta_g"], phys["dt"])
    s.set_lattice(w.get("kappa", 1.0))
    s.set_gravity(1.0, 0.0, 0.0)  # buoyancy along the free stream (aiding flow)
    s.set_bc(2, capi.WALL_DIRICHLET, 1.0)
    s.set_bc(3, capi.FARFIELD)
    s.set_farfield(1.0, phys["uinf"], 0.0, 0.0)
    s.set_state(*st)
    return s, st, (X, Y), phys


def oracle_curv(w):
    """The same cylinder case for the FP64 curvilinear oracle."""
    import oracle
    from oracle import curv as cv
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    X, Y, st, phys = curv_case(inputs, w)
    p = cv.ProblemC(X=X, Y=Y, nu=phys["nu"], chi=phys["chi"], beta_g=phys["beta_g"],
                    dt=phys["dt"], kappa=w.get("kappa", 1.0), gdir=(1.0, 0.0), T_ref=0.0,
                    bc_kind=(cv.PERIODIC, cv.PERIODIC, cv.DIRICHLET, cv.FARFIELD),
                    bc_T=(0.0, 0.0, 1.0, 0.0), inf=(1.0, phys["uinf"], 0.0, 0.0))
    return cv, p, st


def run_curv(args, w):
    """Curvilinear workload: one bench step = `inner` time steps of the cylinder
    O-mesh (one launch per step, graphs), L2 flushed between bench steps."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:  # replicas: one O-mesh per rank, no data-path collective
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    cells = w["ni"] * w["nj"]
    inner = args.inner or w["inner"]
    s, st0, XY, phys = curv_setup(capi, inputs, w)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        s.step(inner)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(inner)
        b.record(stream)
        ev.append((a, b))
    barrier()
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    ms = job_max(sum(a.elapsed_time(b) for a, b in ev))
    value = cells * inner * args.steps * ws / (ms * 1e-3) / 1e6
    host = pinned(st0)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        s.set_state(*host)
        s.step(inner)
        out = s.get_state()
    torch.cuda.synchronize()
    e2e = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    assert np.all(np.isfinite(out[3]))
    heat, perim = s.wall_heat(2)
    nu_cyl = heat * 1.0 / (phys["chi"] * 1.0 * perim)  # Eq. 73 with D = dT = 1
    per_launch = ms * 1e-3 / (inner * args.steps)
    rs = 4 if w["precision"] == "fp32" else 8
    _, ops_cell, sfu_cell = capi.op_counts_curv()
    peak_alu, src = alu_peak(rs)
    alu = ops_cell * cells / per_launch / 1e12
    alg_bytes = 8 * rs * cells
    peak, peak_kind = peaks()
    res, steps_total = s.residual()
    traffic = profile_traffic(args.workload, w["precision"], "curv", CURV_SOURCES)
    line = {
        "metric": "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines",
        "value": round(value, 2), "unit": "M cell-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if rs == 4 else "f64",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "time_steps_per_bench_step": inner, "dt": phys["dt"], "nu": phys["nu"],
                   "l2": "flushed between bench steps (256 MB write)"},
        "e2e": {"value": round(e2e, 2), "unit": "M cell-updates/s",
                "h2d_bytes_per_step": 4 * cells * 8, "d2h_bytes_per_step": 4 * cells * 8},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": round(alu, 3), "peak": round(peak_alu, 3),
                     "unit": "T FP32 op/s" if rs == 4 else "T FP64 op/s",
                     "frac": round(alu / peak_alu, 4), "traffic": traffic,
                     "kernel": "rtlbfsc::curv_step_kernel", "ops_per_cell_update": ops_cell,
                     "sfu_ops_per_cell_update": sfu_cell, "peak_source": src},
        "roofline_hbm": {"bound": "hbm", "achieved": round(alg_bytes / per_launch / 1e9, 1),
                         "peak": peak, "unit": "GB/s",
                         "frac": round(alg_bytes / per_launch / 1e9 / peak, 4), "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs", "alg_bytes_per_launch": alg_bytes},
        "nusselt_cylinder_after_run": round(nu_cyl, 4),
        "clocks": clocks,
        "residual_last_step": res,
    }
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        import oracle
        cv, p, st = oracle_curv(w)
        used = oracle.set_threads(os.cpu_count() or 1)
        n, t0 = 0, time.perf_counter()
        while n == 0 or time.perf_counter() - t0 < args.cpu_seconds:
            st, _, _ = cv.step(p, st, 2)
            n += 2
        dtc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(cells * n / dtc / 1e6, 3), "unit": "M cell-updates/s",
                                "cores": used, "kind": "oracle",
                                "sample": f"{n} FP64 time steps of the same O-mesh ({dtc:.1f} s)"}
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args, w):
    if w.get("kind") == "curv":
        return run_curv(args, w)
    if w.get("kind") == "table6":
        return run_table6(args, w)
    if w.get("kind") == "table4":
        return run_table4(args, w)
    if w.get("kind") == "cavity_tables":
        return run_cavity_tables(args, w)
    if w.get("kind") == "fp64_continue":
        return run_fp64_continue(args, w)
    if w.get("kind") == "cubic":
        return run_cubic(args, w)
    if w.get("kind") == "schemes":
        return run_schemes(args, w)
    if w.get("kind") == "stability":
        return run_stability(args, w)
    if w.get("kind") == "rb_steady":
        return run_rb_steady(args, w)
    if w.get("kind") == "accuracy":
        return run_accuracy(args, w)
    if w.get("kind") == "batch":
        return run_batch(args, w)
    if w.get("kind") == "serve":
        return run_serve(args, w)
    if w.get("kind") == "strips":
        return run_strips(args, w)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, inputs
    capi.lib()
    cells = w["nx"] * w["ny"]
    inner = args.inner or w["inner"]
    s, st0, xf, yf = setup_solver(capi, inputs, w)
    # a dedicated stream shared by torch (events, L2 flush) and the library;
    # the legacy default stream (handle 0) would leave the library on its own
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream)
    # pick the schedule on a snapshot of the state (restored afterwards),
    # or take the one given on the command line
    if args.schedule == "auto":
        sched = s.autotune(max(16, min(256, 2_000_000 // cells + 16)))
    else:
        k = SCHED_NAMES.index(args.schedule.split(":")[0])
        rows = int(args.schedule.split(":")[1]) if ":" in args.schedule else 0
        s.set_schedule(k, rows)
        sched = (k, rows, 0.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        s.step(inner)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    ev = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed iterations (not timed)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(inner)
        b.record(stream)
        ev.append((a, b))
    barrier()
    t_wall = time.perf_counter() - t_wall
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    ms_max = job_max(sum(a.elapsed_time(b) for a, b in ev))
    updates = cells * inner * args.steps * ws
    value = updates / (ms_max * 1e-3) / 1e6

    # e2e through the C ABI with host buffers: the state's cell records
    # (rtlbfs_set_state_raw / get_state_raw, exact, 16 B a cell in FP32),
    # and the four FP64 planes (rtlbfs_set_state / get_state, 32 B a cell
    # plus a conversion kernel each way)
    import numpy as np
    e2e_steps = max(1, min(args.steps, 5))
    rec0, tu0 = s.get_state_raw()
    rec_in = torch.empty(s.raw_bytes(), dtype=torch.uint8, pin_memory=True)
    rec_out = torch.empty(s.raw_bytes(), dtype=torch.uint8, pin_memory=True)
    rec_in.numpy()[...] = rec0
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state_raw(rec_in.numpy(), tu0)
        s.step(inner)
        s.get_state_raw(rec_out.numpy())
    torch.cuda.synchronize()
    e2e = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    bytes_rec = s.raw_bytes()
    host = pinned(st0)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(*host)
        s.step(inner)
        out = s.get_state()
    torch.cuda.synchronize()
    e2e_planes = cells * inner * e2e_steps * ws / job_max(time.perf_counter() - t0) / 1e6
    assert np.all(np.isfinite(out[3]))
    bytes_io = 4 * cells * 8

    rs = 4 if w["precision"] == "fp32" else 8
    per_launch_s = ms_max * 1e-3 / (inner * args.steps)
    kname = SCHED_KERNELS[sched[0]]
    traffic = profile_traffic(args.workload, w["precision"], SCHED_NAMES[sched[0]])
    alu, hbm = rooflines(kname, cells, per_launch_s, rs, traffic, clocks, w.get("scheme", 0))
    res, steps_total = s.residual()
    line = {
        "metric": "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines",
        "value": round(value, 2),
        "unit": "M cell-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if w["precision"] == "fp32" else "f64",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "time_steps_per_bench_step": inner, "parallelism": f"replicas x{ws}",
                   "l2": "flushed between bench steps (256 MB write)",
                   "schedule": {"kernel": SCHED_NAMES[sched[0]], "chunk_rows": sched[1],
                                "autotune_ms_per_step": round(sched[2], 5)},
                   "e2e_host_buffers": "pinned",
                   "state_bytes_per_buffer": 4 * rs * cells},
        "e2e": {"value": round(e2e, 2), "unit": "M cell-updates/s",
                "h2d_bytes_per_step": bytes_rec, "d2h_bytes_per_step": bytes_rec,
                "api": "rtlbfs_set_state_raw / rtlbfs_step / rtlbfs_get_state_raw, pinned"},
        "e2e_planes": {"value": round(e2e_planes, 2), "unit": "M cell-updates/s",
                       "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                       "api": "rtlbfs_set_state / rtlbfs_step / rtlbfs_get_state, pinned"},
        "gpu_launches": int(launches),
        "roofline": alu,
        "roofline_hbm": hbm,
        "clocks": clocks,
        "wall_s": round(t_wall, 3),
        "residual_last_step": res,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if ws > 1:
        torch.distributed.destroy_process_group()
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_strips(args, w):
    """One mesh split by rows over the ranks (strong scaling): rank r steps
    rows split_rows(ny, N)[r] and exchanges its two boundary rows with its
    neighbours before every step (host planes over gloo; the state and the
    residual stay on each GPU).  value = the mesh's cell-updates / the
    slowest rank's device time, exchanges included."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("cpu:gloo,cuda:nccl", device_id=torch.device("cuda", local))
    from paper_2202_13449_gb300 import capi, strips
    capi.lib()
    nx, ny = w["nx"], w["ny"]
    xf = capi.tanh_faces(nx, float(nx), w["phi"])
    yf = capi.tanh_faces(ny, float(ny), w["phi"])
    j0, j1 = strips.split_rows(ny, ws)[rank]
    s = capi.Solver(xf, yf, capi.FP32 if w["precision"] == "fp32" else capi.FP64, rows=(j0, j1))
    dt = 0.5 * float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
    s.set_params(w["Ra"], w["Pr"], w["Ma"], dt)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream)
    sched = s.autotune(16) if args.schedule == "auto" else None
    ex = strips.StripExchange(rank, ws, nx, mode="host", timeout_s=120.0) if ws > 1 else None
    inner = args.inner or w["inner"]
    cells_mine = nx * (j1 - j0)
    state = {"k": 0}

    def steps(n):
        for _ in range(n):
            if ex is not None:
                ex.exchange(s, state["k"])
            s.step(1)
            state["k"] += 1

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        steps(inner)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = capi.launch_count()
    ev = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        steps(inner)
        b.record(stream)
        ev.append((a, b))
    barrier()
    launches = capi.launch_count() - l0
    clocks = clk.stop()
    ms_max = job_max(sum(a.elapsed_time(b) for a, b in ev))
    updates = nx * ny * inner * args.steps
    value = updates / (ms_max * 1e-3) / 1e6
    sums, _ = s.residual_sums()
    res = strips.global_residual(sums)
    # e2e: each rank's strip state up from pinned host buffers and down again
    host = pinned([np.ones((j1 - j0, nx)), np.zeros((j1 - j0, nx)), np.zeros((j1 - j0, nx)),
                   np.tile(1.0 - (0.5 * (xf[1:] + xf[:-1]) / xf[-1]), (j1 - j0, 1))])
    barrier()
    t0 = time.perf_counter()
    for _ in range(2):
        s.set_state(*host)
        state["k"] = 0
        steps(inner)
        out = s.get_state()
    torch.cuda.synchronize()
    e2e = nx * ny * inner * 2 / job_max(time.perf_counter() - t0) / 1e6
    assert np.all(np.isfinite(out[3]))
    per_step_s = ms_max * 1e-3 / (inner * args.steps)
    kname = SCHED_KERNELS[sched[0]] if sched else "rtlbfs::march_kernel"
    alu, hbm = rooflines(kname, cells_mine, per_step_s, 4, None, clocks)
    line = {
        "metric": "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines",
        "value": round(value, 2), "unit": "M cell-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": nx * ny,
                   "time_steps_per_bench_step": inner,
                   "parallelism": f"row strips x{ws} (2-row halo exchange per step, gloo)",
                   "rows_rank0": list(strips.split_rows(ny, ws)[0]),
                   "l2": "flushed between bench steps (256 MB write)",
                   "schedule": ({"kernel": SCHED_NAMES[sched[0]], "chunk_rows": sched[1]}
                                if sched else args.schedule)},
        "e2e": {"value": round(e2e, 2), "unit": "M cell-updates/s",
                "h2d_bytes_per_step": 32 * nx * ny, "d2h_bytes_per_step": 32 * nx * ny},
        "gpu_launches": int(job_sum(launches)),
        "roofline": alu, "roofline_hbm": hbm,
        "roofline_note": "per GPU, its strip's cell-updates over the job's time per step "
                         "(halo exchanges included)",
        "clocks": clocks,
        "residual_last_step": list(res),
    }
    if ws > 1:
        torch.distributed.destroy_process_group()
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def oracle_problem(oracle, inputs, w):
    import numpy as np
    nx, ny = w["nx"], w["ny"]
    if w["kind"] in ("cavity", "strips"):
        xf = oracle.tanh_faces(nx, float(nx), w["phi"])
        yf = oracle.tanh_faces(ny, float(ny), w["phi"])
        nu, chi, bg = oracle.params_from_ra(w["Ra"], w["Pr"], w["Ma"], float(nx))
        dt = 0.5 * float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
        p = oracle.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=bg, dt=dt)
        st = inputs.conduction_state(xf, yf)
    else:
        xf, yf = inputs.uniform_faces(nx), inputs.uniform_faces(ny)
        nu, chi, bg = oracle.params_from_ra(w["Ra"], w["Pr"], w["Ma"], float(ny))
        p = oracle.Problem(xf=xf, yf=yf, nu=nu, chi=chi, beta_g=bg, dt=0.5,
                           bc_kind=(oracle.PERIODIC, oracle.PERIODIC, oracle.DIRICHLET,
                                    oracle.DIRICHLET), bc_T=(0, 0, 1, 0))
        st = inputs.rb_state(xf, yf, amp=1e-3, seed=0)
    return p, st


def cpu_baseline(w, seconds):
    """The FP64 oracle as it stands on this host's cores, on a bounded sample
    of the same workload (time steps of the same mesh until `seconds`)."""
    import oracle
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    p, st = oracle_problem(oracle, inputs, w)
    cells = w["nx"] * w["ny"]
    st, _, _ = oracle.step(p, st, 1)  # warm
    n, t0 = 0, time.perf_counter()
    chunk = 2
    while time.perf_counter() - t0 < seconds:
        st, _, _ = oracle.step(p, st, chunk)
        n += chunk
    dt = time.perf_counter() - t0
    return {"value": round(cells * n / dt / 1e6, 3), "unit": "M cell-updates/s", "cores": used,
            "kind": "oracle",
            "sample": f"{n} FP64 time steps of the same {w['nx']}x{w['ny']} mesh "
                      f"({dt:.1f} s, OpenMP over rows)"}


def auto_dt(xf, yf, nu, chi):
    """The library's stability rule for dt = 0: min(w/2, 0.2 w^2 / max(nu, chi))."""
    import numpy as np
    wmin = float(min(np.min(np.diff(xf)), np.min(np.diff(yf))))
    return min(0.5 * wmin, 0.2 * wmin * wmin / max(nu, chi))


def batch_problems(oracle, inputs, w, count):
    """Oracle problems of the first `count` cavities of the batch workload."""
    out = []
    for sp in inputs.batch_specs(w["count"], w["seed"])[:count]:
        xf = oracle.tanh_faces(sp.n, float(sp.n), sp.phi)
        nu, chi, bg = oracle.params_from_ra(sp.Ra, sp.Pr, 0.1, float(sp.n))
        p = oracle.Problem(xf=xf, yf=xf, nu=nu, chi=chi, beta_g=bg, dt=auto_dt(xf, xf, nu, chi))
        out.append((p, inputs.conduction_state(xf, xf), sp.n * sp.n))
    return out


def request_problem(oracle, inputs, n, Ra, Pr):
    xf = inputs.uniform_faces(n)
    nu, chi, bg = oracle.params_from_ra(Ra, Pr, 0.1, float(n))
    p = oracle.Problem(xf=xf, yf=xf, nu=nu, chi=chi, beta_g=bg, dt=auto_dt(xf, xf, nu, chi))
    return p, inputs.conduction_state(xf, xf)


def cpu_baseline_batch(w, seconds):
    """The FP64 oracle on the first cavities of the batch, a few steps each,
    round after round until `seconds` have passed."""
    import oracle
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    used = oracle.set_threads(os.cpu_count() or 1)
    probs = batch_problems(oracle, inputs, w, 16)
    states = [st for _, st, _ in probs]
    updates, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for k, (p, _, cells) in enumerate(probs):
            states[k], _, _ = oracle.step(p, states[k], 2)
            updates += 2 * cells
    dt = time.perf_counter() - t0
    return {"value": round(updates / dt / 1e6, 3), "unit": "M cell-updates/s", "cores": used,
            "kind": "oracle",
            "sample": f"the first 16 cavities of the batch, 2 FP64 steps each per round, "
                      f"{updates / 1e6:.1f} M cell-updates in {dt:.1f} s (OpenMP over rows)"}


def oracle_solve_estimate(oracle, inputs, n, Ra, Pr, steps_needed, probe_steps=2):
    """Seconds the oracle would take for one request: probe_steps timed
    steps, scaled to the steps the request needs."""
    p, st = request_problem(oracle, inputs, n, Ra, Pr)
    t0 = time.perf_counter()
    oracle.step(p, st, probe_steps)
    return (time.perf_counter() - t0) / probe_steps * steps_needed


def cpu_baseline_serve(w, reqs, steps_by_req, seconds):
    """Oracle solves/s for the trace's requests in arrival order, each timed
    for 2 steps and scaled to the step count the GPU run gave it (or the cap),
    until `seconds` of probing have passed."""
    import oracle
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    used = oracle.set_threads(os.cpu_count() or 1)
    est, k, t0 = 0.0, 0, time.perf_counter()
    cap = steps_by_req if isinstance(steps_by_req, int) else None
    while k < len(reqs) and time.perf_counter() - t0 < seconds:
        _, n, Ra, Pr = reqs[k]
        need = cap if cap is not None else max(1, int(steps_by_req[k]))
        est += oracle_solve_estimate(oracle, inputs, n, Ra, Pr, need)
        k += 1
    return {"value": round(k / est, 5) if est > 0 else None, "unit": "solves/s", "cores": used,
            "kind": "oracle",
            "sample": f"the first {k} requests of the trace, each timed for 2 FP64 steps and "
                      f"scaled to its step count (extrapolated: {est:.0f} s of oracle work)"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2202_13449_gb300 import inputs
    oracle.build()
    used = oracle.set_threads(os.cpu_count() or 1)
    per_step = max(1, int(args.ref_steps_per_step))
    kind = w.get("kind")
    if kind == "serve":
        # each bench step: the next request of the trace, probed for 2 steps
        # and scaled to the steps it needs: the step cap, or for a sub-trace
        # whose requests converge, the estimate of the thermal diffusion time
        # 10 N sqrt(Ra Pr) / Delta t (Delta t = 0.5 on these unit-cell meshes)
        # when that is below the cap
        trace = inputs.serving_trace(w["count"], w["seed"], w["rate"])
        trace = [r for r in trace
                 if r.n <= w.get("n_max", r.n) and r.Ra <= w.get("ra_max", r.Ra)]
        reqs = [(r.t_arrive, r.n, r.Ra, r.Pr) for r in trace]
        cap = w.get("max_steps", 2000) if args.max_steps is None else args.max_steps

        def need(q):
            if "n_max" not in w:
                return cap
            return int(min(cap, 10 * q[1] * (q[2] * q[3]) ** 0.5 / 0.5))

        for k in range(args.warmup):
            q = reqs[k % len(reqs)]
            oracle_solve_estimate(oracle, inputs, *q[1:], need(q))
        est = 0.0
        for k in range(args.steps):
            q = reqs[k % len(reqs)]
            est += oracle_solve_estimate(oracle, inputs, *q[1:], need(q))
        value = args.steps / est
        line = {
            "impl": "reference",
            "metric": "batched solves/s and p50/p99 time-to-steady (request loop)",
            "value": round(value, 5), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(est * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": args.workload, "description": w["desc"],
                       "max_steps_cap": cap,
                       "note": "reference arm = the FP64 CPU oracle (the paper ships no code); "
                               "one request per bench step, extrapolated from 2 timed steps"},
            "e2e": {"value": round(value, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "cpu_baseline": {"value": round(value, 5), "unit": "solves/s", "cores": used,
                             "kind": "oracle",
                             "sample": f"the first {args.steps} requests of the trace, 2 timed "
                                       f"FP64 steps each, scaled to "
                                       + ("10 N sqrt(Ra Pr) / 0.5 steps (at most the cap)"
                                          if "n_max" in w else f"{cap} steps")},
        }
        print(json.dumps(line), flush=True)
        return
    if kind == "stability":
        probs = []
        for nn, ra, ka in stability_cases(w)[:8]:
            p = oracle.cavity_problem(nn, ra, dt=w["dt"])
            p.kappa = ka
            probs.append((p, inputs.conduction_state(p.xf, p.yf), nn * nn))
        states = [st for _, st, _ in probs]
        cells = sum(c for _, _, c in probs)

        def one():
            for k, (p, _, _) in enumerate(probs):
                states[k], _, _ = oracle.step(p, states[k], per_step)
        sample = f"the first 8 cases of the map ({cells} cells), {per_step} FP64 steps each"
    elif kind == "batch":
        probs = batch_problems(oracle, inputs, w, 16)
        states = [st for _, st, _ in probs]
        cells = sum(c for _, _, c in probs)

        def one():
            for k, (p, _, _) in enumerate(probs):
                states[k], _, _ = oracle.step(p, states[k], per_step)
        sample = f"the first 16 cavities of the batch ({cells} cells), {per_step} FP64 steps each"
    elif kind == "curv":
        cv, p, st0 = oracle_curv(w)
        cells = w["ni"] * w["nj"]
        box = [st0]

        def one():
            box[0], _, _ = cv.step(p, box[0], per_step)
        sample = f"{per_step} FP64 time steps of the {w['ni']}x{w['nj']} O-mesh"
    elif kind == "cubic":
        _, d3, p, st0 = oracle_cubic(w)
        cells = w["n"] ** 3
        box = [st0]

        def one():
            box[0], _, _ = d3.step(p, box[0], per_step)
        sample = f"{per_step} FP64 time steps of the {w['n']}^3 mesh"
    else:
        p, st0 = oracle_problem(oracle, inputs, w)
        cells = w["nx"] * w["ny"]
        box = [st0]

        def one():
            box[0], _, _ = oracle.step(p, box[0], per_step)
        sample = f"{per_step} FP64 time steps of the {w['nx']}x{w['ny']} mesh"
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = cells * per_step * args.steps / dt / 1e6
    metric = ("stability map: M cell-updates/s of the batched cases (wall time of the call)"
              if kind == "stability" else
              "M cell-updates/s (whole job) and fraction of the ALU and HBM rooflines")
    line = {
        "impl": "reference",
        "metric": metric,
        "value": round(value, 3), "unit": "M cell-updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "description": w["desc"], "cells": cells,
                   "time_steps_per_bench_step": per_step,
                   "note": "reference arm = the FP64 CPU oracle (the paper ships no code)"},
        "e2e": {"value": round(value, 3), "unit": "M cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": round(value, 3), "unit": "M cell-updates/s", "cores": used,
                         "kind": "oracle", "sample": f"{args.steps} x {sample}"},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", type=int, default=0, help="time steps per bench step")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-steps-per-step", type=int, default=4)
    ap.add_argument("--max-steps", type=int, default=None,
                    help="serve: step cap per request (default: the workload's, else 2000)")
    ap.add_argument("--tol", type=float, default=None,
                    help="serve: steady tolerance (default: the workload's, else 1e-7; keep it "
                         "above the FP32 residual floor ~1.4e-8)")
    ap.add_argument("--time-limit", type=float, default=None,
                    help="serve: wall-clock cap in s (default: the workload's, else 60)")
    ap.add_argument("--slots", type=int, default=256, help="serve: concurrent cavities")
    ap.add_argument("--fp64-sample", type=int, default=20, help="serve: FP64 comparator sample")
    ap.add_argument("--schedule", default="auto",
                    help="auto (autotuner), or march|tile|persist[:rows per unit or tile]")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        if w.get("kind") in ("accuracy", "rb_steady", "schemes", "table6", "table4",
                             "cavity_tables", "fp64_continue"):
            print(json.dumps({"impl": "reference", "unavailable": "this run measures accuracy or "
                              "time to a steady state of the GPU path; the oracle's rate is the "
                              "rb1024x512 / cavity512 reference lines"}))
            return
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
