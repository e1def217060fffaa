#!/usr/bin/env python3
"""Throughput of one time step of the Fourier spectral FFT+CG splitting scheme
for the periodic Hu-Cai system (arXiv 2606.06720, Algorithm 1) on GB300.

Workload: the 2048^2 source/sink problem (smooth random r in [0.05, 0.15],
S = +G(0.3,0.5) - G(0.7,0.5) with sigma 0.05, m0 ~ U[0, 0.5], c = 25,
D = 0.02, gamma = 0.5, dt = 5e-4), FP32 operator/FFT/split step with the
pressure solve wrapped in FP64 iterative refinement to a relative residual of
1e-8.  A "step" is one pass of the loop body of Algorithm 1 (pressure solve +
activation + relaxation + diffusion).  Metric: Mpoint-steps/s = nx*ny*steps /
time / 1e6, summed over ranks (each rank runs an independent replica).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (the reference arm; see cpu_baseline).  `--accuracy` runs the
equal-accuracy calibration of the plain FP64 path and prints its summary.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoint-steps/s at 2048² FP32-refined vs FP64 plain at equal accuracy; HBM GB/s"
UNIT = "Mpoint-steps/s"
N_GRID = 2048
CG_RTOL_REFINED = 1e-8      # the refined path's pressure tolerance
FP64_EQUAL_RTOL = 1e-4      # loosest plain-FP64 tolerance reaching m rel. L2 <= 1e-5 at 100 steps
# Preconditioner of the timed legs: the anisotropic option of reading R3
# (-div(Kbar grad), Kbar = mean(m m^T) + mean(r) I).  It changes CG iteration
# counts only; the library's default, kappa (-Laplacian), is the scalar_kappa leg.
PRECOND = "kbar"
                            # (calibrated with --accuracy: rtol 1e-4 gives 5.9e-7, 1e-3 gives 2.2e-5)
HBM_PEAK_FALLBACK = 6800.0  # GB/s, recipe fallback when MEASURED_PEAKS.json is absent
FP64_PEAK_NOMINAL = 1.25    # TFLOP/s, nominal FP64 of GB300 (recipe table): context only; the
                            # FP64 kernels are reported against the measured FMA peak
                            # (hc_fp64_fma_peak) taken in the same run

# Algorithmic bytes moved per launch of each step kernel, in units of n = nx*ny
# points (F4 = 4n bytes: one FP32 field, physical or packed spectral; F8 = 8n).
# Each input read once, each output written once; scalars and tables ignored.
BYTES_PER_POINT = {
    "fp32_refined": {
        "cg_grad": 20,     # read r, d; write d, Gx, Gy          5 F4
        "cg_apply": 28,    # read Gx, Gy, mx, my, r; write Qx, Qy 7 F4
        "cg_div": 12,      # read Qx, Qy; write q                 3 F4 (alpha comes from cg_apply)
        "cg_update": 24,   # read x, r, d, q; write x, r          6 F4
        "res_grad": 24,    # read p64; write Gx64, Gy64           3 F8
        "res_apply": 44,   # read Gx64, Gy64 (2 F8), m, r (3 F4); write 2 F8
        "res_div": 40,     # read Qx64, Qy64, b64; write r64 (4 F8) + r32, delta (2 F4)
        "split_grad": 16,  # read p64 (F8); write Gx, Gy (2 F4)
        "split_row": 24,   # read Gx, Gy, mx, my; write Mx, My    6 F4
        "split_heat": 16,  # read Mx, My; write Mx, My            4 F4
        "split_c2r": 16,   # read Mx, My; write mx, my            4 F4
        "first_grad": 16,  # read p64 (F8); write Gx, Gy (2 F4)
        "first_apply": 28, # read Gx, Gy, mx, my, r; write Qx, Qy  7 F4
        "first_div": 20,   # read Qx, Qy, b32; write r32, delta   5 F4
        "mid_grad": 24,    # as res_grad (double-float grads are F8 too)
        "mid_apply": 44,   # as res_apply
        "mid_div": 32,     # read Qx, Qy, b (3 F8); write r32, delta (2 F4)
    },
    "fp64": {
        "cg_grad": 40, "cg_apply": 56, "cg_div": 24, "cg_update": 48, "res_grad": 24,
        "res_apply": 56, "res_div": 32, "split_grad": 24, "split_row": 48, "split_heat": 32,
        "split_c2r": 32,
    },
}
FP64_KERNELS = {"fp32_refined": {"res_grad", "res_apply", "res_div", "res_ypass"},
                "fp64": set(BYTES_PER_POINT["fp64"])}
# Double-float kernels (the mid-step residual of the FP64-refined path): bound
# by the FP32 pipes running the emulated arithmetic; no roofline fraction.
DF_KERNELS = {"mid_grad", "mid_apply", "mid_div", "mid_ypass"}

# The 3D kernels (d = 3, n = nx*ny*nz points), refined path, same convention.
# The y pass runs twice per operator apply (inverse before the row pass,
# forward after it); split_heat / split_c2r are the y / z diffusion passes.
BYTES_PER_POINT_3D = {
    "cg_grad": 24,     # read r, d; write d, G0, G1, G2        6 F4
    "cg_ypass": 24,    # read G0..G2; write G0..G2             6 F4
    "cg_apply": 40,    # read G0..G2, m0..m2, r; write Q0..Q2 10 F4
    "cg_div": 16,      # read Q0..Q2; write q                  4 F4
    "cg_update": 24,   # read x, r, d, q; write x, r           6 F4
    "res_grad": 44,    # read p64, delta; write p64, 3 grads (F8)
    "res_ypass": 48,   # 3 F8 in, 3 F8 out
    "res_apply": 64,   # read 3 F8 + 4 F4; write 3 F8
    "res_div": 48,     # read 3 F8 + b64; write r64 (F8), r32, delta (F4)
    "split_grad": 20,  # read p64 (F8); write 3 F4
    "split_row": 36,   # read 3 grads, 3 m; write 3 m          9 F4
    "split_heat": 24,  # y diffusion of m in place             6 F4
    "split_c2r": 24,   # z diffusion of m in place + sum |m|^2 6 F4
    "first_grad": 20,  # read p64 (F8); write 3 F4
    "first_apply": 40, # as cg_apply
    "first_div": 24,   # read Q0..Q2, b32; write r32, delta  6 F4
    "mid_grad": 44,    # as res_grad
    "mid_ypass": 48,   # as res_ypass
    "mid_apply": 64,   # as res_apply
    "mid_div": 40,     # read 3 F8 + b (F8); write r32, delta (F4)
}

# DRAM bytes (read + write) per launch measured by ncu for the 2048^2 refined
# workload with the current kernels (from the committed ncu summaries).
# Set an entry to None when its kernel changes.
NCU_TRAFFIC_2048 = {"res_grad": 104.6e6, "res_apply": 132.7e6, "res_div": 132.7e6,
                    "cg_grad": 19.4e6, "cg_apply": 86.8e6, "cg_div": 34.1e6, "cg_update": 67.8e6,
                    "split_grad": 37.2e6, "split_heat": 33.7e6, "split_c2r": 34.1e6,
                    "first_grad": 37.2e6, "first_div": 52.4e6,
                    "mid_grad": None, "mid_apply": None, "mid_div": None, "split_row": None}


def shard(items: int, rank: int, world: int) -> list:
    """Indices of the independent problems rank `rank` runs (round robin)."""
    return [i for i in range(items) if i % world == rank]


def aggregate(local_ms: float, local_units: float, world: int, reduce_max, reduce_sum):
    """Whole-job throughput from per-rank timings: the slowest rank's time and
    the units all ranks processed.  Returns (max_ms, units_total, units per
    second)."""
    ms = reduce_max(local_ms) if world > 1 else local_ms
    units = reduce_sum(local_units) if world > 1 else local_units
    return ms, units, units / (ms / 1e3)


def fft_flops_per_point(kernel: str, nx: int, ny: int) -> float:
    """Algorithmic FLOPs per point and launch: 5 N log2 N per complex FFT of
    length N (the usual FFT count), plus the pointwise algebra."""
    lx, ly = math.log2(nx), math.log2(ny)
    col2 = 5.0 * ly            # two length-ny complex FFTs over nx/2 columns
    row1 = 5.0 * lx            # one length-nx complex FFT per row
    return {
        "cg_grad": col2 + 4, "res_grad": col2 + 2, "split_grad": col2 + 2,
        "cg_apply": 2 * row1 + 9, "res_apply": 2 * row1 + 9,
        "cg_div": col2 + 6, "res_div": col2 + 10,
        "cg_update": 10, "split_row": 2 * row1 + 30, "split_heat": 2 * col2 + 3,
        "split_c2r": row1 + 2, "first_grad": col2 + 2, "first_apply": 2 * row1 + 9,
        "first_div": col2 + 10, "mid_grad": col2 + 2, "mid_apply": 2 * row1 + 9,
        "mid_div": col2 + 10,
    }[kernel]


def fft_flops_per_point_3d(kernel: str, nx: int, ny: int, nz: int) -> float:
    """As fft_flops_per_point for the 3D kernels: column passes do three
    complex FFTs per packed column (n/2 columns of length L: 7.5 log2 L per
    point), the row-pair passes three complex row FFTs per pair of rows in
    each direction (15 log2 nx per point)."""
    lx, ly, lz = math.log2(nx), math.log2(ny), math.log2(nz)
    return {
        "cg_grad": 7.5 * lz + 6, "res_grad": 7.5 * lz + 4, "split_grad": 7.5 * lz + 3,
        "cg_ypass": 7.5 * ly, "res_ypass": 7.5 * ly,
        "cg_apply": 15 * lx + 11, "res_apply": 15 * lx + 11,
        "cg_div": 7.5 * lz + 8, "res_div": 7.5 * lz + 12, "cg_update": 10,
        "split_row": 30 * lx + 45, "split_heat": 15 * ly + 3, "split_c2r": 15 * lz + 5,
        "first_grad": 7.5 * lz + 3, "first_apply": 15 * lx + 11, "first_div": 7.5 * lz + 12,
        "mid_grad": 7.5 * lz + 4, "mid_ypass": 7.5 * ly, "mid_apply": 15 * lx + 11,
        "mid_div": 7.5 * lz + 12,
    }[kernel]


def kernel_table(s, counts: dict, bytes_pp: dict, flops_pp, fp64_names: set, npts: int,
                 reps: int, hbm_peak: float, fp64_peak: float) -> dict:
    """Per-kernel CUDA-event durations (hc_time_kernel: back-to-back launches
    on the same data) with algorithmic GB/s and TFLOP/s and the fraction of
    the kernel's roof: HBM for the FP32 kernels, the measured FP64 FMA peak
    for the FP64 ones."""
    kernels = {}
    for name, cnt in counts.items():
        kms = s.time_kernel(name, reps=reps)
        gbs = bytes_pp[name] * npts / (kms / 1e3) / 1e9
        tfl = flops_pp(name) * npts / (kms / 1e3) / 1e12
        is64 = name in fp64_names
        isdf = name in DF_KERNELS
        kernels[name] = {"ms": kms, "launches_per_step": cnt, "ms_per_step": kms * cnt,
                         "alg_GBs": gbs, "alg_TFLOPs": tfl,
                         "bound": "alu-df" if isdf else ("alu" if is64 else "hbm"),
                         "frac": None if isdf else ((tfl / fp64_peak) if is64
                                                    else (gbs / hbm_peak))}
    return kernels


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) taken while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str, path: str = None):
        """path: where the raw samples go (kept); default a temporary file."""
        self.gpu_id = gpu_id
        self.proc = None
        if path is None:
            import tempfile
            path = os.path.join(tempfile.gettempdir(), f"hc_bench_clocks_{os.getpid()}.csv")
        self.path = path

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                          if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------- oracle (CPU)
def oracle_steps(n: int, steps: int, warm: int = 1):
    """Time `steps` oracle steps of the source/sink workload resampled at n^2,
    after `warm` untimed steps (so the timed steps are warm-started like the
    GPU's), with the preconditioner the GPU legs use.  Returns (seconds,
    threads, cg_iters)."""
    import numpy as np
    import oracle as O
    import workloads as W
    threads = os.cpu_count() or 1
    O.set_threads(threads)
    w = W.source_sink_2d(n)
    g = O.Grid(w.n, w.L)
    prm = O.Params(c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, cg_rtol=CG_RTOL_REFINED, cg_maxit=2000,
                   precond=1 if PRECOND == "kbar" else 0)
    m, p = w.m0.copy(), np.zeros(g.shape)
    for _ in range(warm):
        m, p, _ = O.step(g, prm, w.r, w.S, m, p)
    t0 = time.perf_counter()
    iters = 0
    for _ in range(steps):
        m, p, st = O.step(g, prm, w.r, w.S, m, p)
        iters += st.cg_iters
    return time.perf_counter() - t0, threads, iters


def workload_config(extra: dict | None = None) -> dict:
    cfg = {
        "workload": "source_sink_2048: 2048x2048 periodic unit square, smooth random r in "
                    "[0.05,0.15] (|k|<=8, seed 0), S=+G(0.3,0.5)-G(0.7,0.5) sigma 0.05 minus mean, "
                    "m0~U[0,0.5] seed 0, c=25 D=0.02 gamma=0.5 dt=5e-4",
        "precision": "FP32 FFT/operator/split step + FP64 iterative refinement of the pressure",
        "cg_rtol": CG_RTOL_REFINED,
        "preconditioner": "kbar: -div(Kbar grad), Kbar = mean(m m^T) + mean(r) I (reading R3's "
                          "anisotropic option; the default scalar kappa is the scalar_kappa leg)",
        "grid": [N_GRID, N_GRID],
        "l2": "inputs larger than L2 (refined working set ~390 MB > 129 MiB L2); no flush",
        "loop_control": "one CUDA graph per step, CG/refinement loops as conditional WHILE nodes",
        "parallelism": "replicas (one independent problem per GPU)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------- reference arm
def reference_grid(steps: int) -> int:
    """The reference arm's sample grid: the 2048^2 workload itself when its
    oracle steps fit a few minutes (about 7 s per step on 16 cores), else the
    same workload resampled at 1024^2 or 512^2."""
    return N_GRID if steps <= 20 else (1024 if steps <= 80 else 512)


def run_reference(args) -> None:
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = args.ref_n or reference_grid(args.steps)
    K, Wm = args.steps, args.warmup
    secs, threads, iters = oracle_steps(n, K, warm=max(min(Wm, 3), 1))
    value = n * n * K / secs / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": Wm, "ms_per_step": secs / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config({"precision": "FP64 (the CPU oracle)",
                                   "sample_grid": [n, n]}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"the same workload at {n}x{n}; each timed step is one FP64 "
                                   f"oracle step (warm-started, cg_rtol {CG_RTOL_REFINED}, the "
                                   f"Kbar preconditioner of the GPU legs)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cg_iters_per_step": iters / K,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- accuracy calibration
def run_accuracy(args) -> None:
    """The equal-accuracy calibration on its own, with more tolerances and
    each leg's throughput."""
    import torch
    import workloads as W
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2606_06720_gb300 as P
    out = equal_accuracy(P, W, torch.device("cuda", 0), args.acc_steps,
                         [("fp32_refined", CG_RTOL_REFINED), ("fp32_refined_df", CG_RTOL_REFINED),
                          ("fp64", 1e-3), ("fp64", 1e-4), ("fp64", 1e-5), ("fp64", 1e-6)],
                         timed=True)
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- diagnostics leg
def run_diagnostics(P, W, args, dev, barrier, job_rate, headline) -> dict:
    """(a) The headline 2048^2 workload with the energy and Delta m computed
    every step, run as Algorithm 1's loop (hc_run: eps 1e-4, energy rule on;
    neither fires within the steps timed): its throughput against the
    headline's.  (b) The paper's own setups of Sections 3.2-3.3 at 512^2
    (c = 200, D = 0.0025, dt = 0.005, CG threshold 1e-7 relative): one source
    and four sinks from m^A (gamma = 1), and the internal sink from m^const
    (gamma = 0.75), each run through hc_run."""
    import numpy as np
    import torch
    out = {}
    w = W.source_sink_2d(N_GRID)
    K = max(10, args.steps // 10)
    s = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp32_refined",
                 cg_rtol=CG_RTOL_REFINED, cg_maxit=2000, precond=PRECOND,
                 device=str(dev), diagnostics=True)
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    s.run(3, eps=1e-4)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = s.run(K, eps=1e-4, stop_on_energy=True)
    torch.cuda.synchronize()
    _, v = job_rate((time.perf_counter() - t0) * 1e3, w.npts * st.steps)
    s.close()
    out["headline_with_diagnostics"] = {
        "value": v, "unit": UNIT, "steps": st.steps, "stop_reason": st.stop_reason,
        "cost_vs_headline": headline / v - 1.0, "energy": st.energy, "delta_m": st.delta_m,
        "path": "hc_run (gated step graph, host checks every 16 launches)"}
    for name, wp in (("paper_four_sinks_512_gamma1", W.paper_four_sinks(512, 1.0)),
                     ("paper_internal_sink_512_mconst", W.paper_internal_sink(512, 0.75))):
        sp = P.Solver(wp.n, wp.L, c=wp.c, D=wp.D, gamma=wp.gamma, dt=wp.dt,
                      precision="fp32_refined", cg_rtol=wp.cg_rtol, cg_maxit=2000, precond=PRECOND,
                      device=str(dev))
        sp.set_r(wp.r)
        sp.set_source(wp.S)
        sp.set_m(wp.m0)
        Kp = max(20, args.steps // 5)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stp = sp.run(Kp, eps=1e-4, stop_on_energy=True)
        torch.cuda.synchronize()
        _, vp = job_rate((time.perf_counter() - t0) * 1e3, wp.npts * stp.steps)
        sp.close()
        out[name] = {"value": vp, "unit": UNIT,
                     "steps": stp.steps, "t_end": stp.steps * wp.dt,
                     "stop_reason": stp.stop_reason, "energy": stp.energy,
                     "delta_m": stp.delta_m, "cg_iters_last_step": stp.cg_iters}
    return out


# ----------------------------------------------------------------- paper's convergence grids
# Section 4's first grid-convergence table at t = 5 (context only: these are
# the paper's long-run CPU figures, parity unpinned).
PAPER_Q_T5 = {"50-100-200": {"q_m": 6.6747, "q_grad_p": 5.0983, "q_p": 5.6516},
              "100-200-400": {"q_m": 3.9922, "q_grad_p": 3.8377, "q_p": 3.2919},
              "200-400-800": {"q_m": 3.4010, "q_grad_p": 4.5286, "q_p": 5.6811}}


def run_convergence(P, W, args, dev, job_rate) -> dict:
    """The paper's grid-convergence setup (S_int, m^A, c = 100, gamma = 0.75,
    D = 0.01, dt = 0.05, CG threshold 1e-7) on N = 50, 100, 200, 400, 800, the
    mixed-radix FP64 path, to t = 5 (100 steps).  The observed orders
    q = ln(|u_h - u_h/2| / |u_h/2 - u_h/4|) / ln 2 of Section 4 for u = |m|,
    |grad p| and p, with the finer solutions sampled at the coarse nodes
    (every second node), beside the paper's values; and each run's throughput."""
    import numpy as np
    import torch
    sizes = (50, 100, 200, 400, 800)
    K = args.conv_steps
    sol, rate, iters = {}, {}, {}
    for n in sizes:
        w = W.paper_convergence(n, steps=K)
        with P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp64",
                      cg_rtol=w.cg_rtol, cg_maxit=5000, precond=PRECOND, device=str(dev)) as s:
            s.set_r(w.r)
            s.set_source(w.S)
            s.set_m(w.m0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = s.step(K)
            torch.cuda.synchronize()
            _, rate[n] = job_rate((time.perf_counter() - t0) * 1e3, w.npts * K)
            iters[n] = st.total_cg_iters / K
            m, p, gp = s.get_m(), s.get_p(), s.gradient().reshape((2,) + w.shape)
        sol[n] = {"m": np.sqrt((m.reshape((2,) + w.shape) ** 2).sum(0)), "grad_p": np.sqrt((gp ** 2).sum(0)),
                  "p": p}

    def diff(a, b):  # b on the grid twice as fine, sampled at a's nodes
        return float(np.linalg.norm(a - b[::2, ::2]))

    orders = {}
    for n in sizes[:-2]:
        key = f"{n}-{2 * n}-{4 * n}"
        orders[key] = {
            "q_" + f: math.log(diff(sol[n][f], sol[2 * n][f]) / diff(sol[2 * n][f], sol[4 * n][f]))
            / math.log(2.0) for f in ("m", "grad_p", "p")}
    return {"t": K * 0.05, "steps": K, "grids": list(sizes), "orders": orders,
            "paper_orders_t5": PAPER_Q_T5 if K == 100 else None,
            "mpoint_steps_per_s": {str(n): rate[n] for n in sizes},
            "cg_iters_per_step": {str(n): iters[n] for n in sizes},
            "path": "mixed-radix FP64 kernels (radix 4, 2, 5 passes); Kbar preconditioner; "
                    "context only, parity unpinned (the paper's long-run figures)"}


# ----------------------------------------------------------------- 3D leg
def run_3d(P, W, args, dev, barrier, job_rate, hbm_peak, hbm_src, fp64_peak) -> dict:
    """The 256^3 source/sink workload (r = 0.1, sigma 0.05 pair at
    (0.3,0.5,0.5)/(0.7,0.5,0.5), m0 ~ U[0,0.5], c = 25, D = 0.03,
    gamma = 0.75, dt = 5e-4), FP32 + FP64 refinement to 1e-8, graph mode."""
    import numpy as np
    import torch
    w = W.source_sink_3d(args.n3d)
    s = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp32_refined",
                 cg_rtol=CG_RTOL_REFINED, cg_maxit=2000, precond=PRECOND,
                 use_graph=not args.host_loop,
                 device=str(dev))
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    s.step(max(args.warmup, 3) if args.only_3d else 3)
    K3 = args.steps if args.only_3d else max(5, args.steps // 30)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed3d")
    e0.record(s.stream)
    st = s.step(K3)
    e1.record(s.stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    npts = w.npts
    ms, value = job_rate(e0.elapsed_time(e1), npts * K3)
    it = st.total_cg_iters / K3
    sw = st.total_sweeps / K3
    r64 = st.total_refine_residuals / K3  # FP64 residuals per step
    mid = st.total_mid_df / K3           # double-float mid-step residuals per step
    counts = {"cg_grad": it, "cg_ypass": 2 * it, "cg_apply": it, "cg_div": it, "cg_update": it,
              "res_grad": r64, "res_ypass": 2 * r64, "res_apply": r64, "res_div": r64,
              "split_grad": 1, "split_row": 1, "split_heat": 1, "split_c2r": 1,
              "first_grad": 1, "first_apply": 1, "first_div": 1}
    if mid > 0:
        counts.update({"mid_grad": mid, "mid_ypass": 2 * mid, "mid_apply": mid, "mid_div": mid})
    kernels = kernel_table(s, counts, BYTES_PER_POINT_3D,
                           lambda k: fft_flops_per_point_3d(k, *w.n),
                           FP64_KERNELS["fp32_refined"], npts, max(3, args.kernel_reps // 3),
                           hbm_peak, fp64_peak)
    s.close()
    # dominant FP32 kernel of the CG iteration against HBM
    fp32 = [k for k in kernels if kernels[k]["bound"] == "hbm"]
    dom = max(fp32, key=lambda k: kernels[k]["ms_per_step"])
    dk = kernels[dom]
    plain = None if args.no_fp64 else run_3d_fp64_plain(P, W, args, dev, barrier, job_rate, K3, value)
    return {"value": value, "unit": UNIT, "ms_per_step": ms / K3,
            "steps": K3, "grid": list(w.n),
            "workload": "source_sink_3d_%d: r=0.1, S=+G(0.3,0.5,0.5)-G(0.7,0.5,0.5) sigma 0.05 "
                        "minus mean, m0~U[0,0.5] seed 0, c=25 D=0.03 gamma=0.75 dt=5e-4; "
                        "FP32 + FP64 refinement, cg_rtol 1e-8" % args.n3d,
            "cg_iters_per_step": it, "refine_sweeps_per_step": sw,
            "fp64_residuals_per_step": r64, "df_mid_residuals_per_step": mid,
            "rel_residual_last_step": st.rel_residual,
            "roofline_fp32": {"bound": "hbm", "kernel": dom, "achieved": dk["alg_GBs"],
                              "peak": hbm_peak, "unit": "GB/s", "frac": dk["frac"],
                              "peak_source": hbm_src,
                              "alg_bytes": BYTES_PER_POINT_3D[dom] * npts},
            "fp64_plain": plain,
            "kernels": kernels}


# Plain-FP64 tolerances tried for the 3D comparison, loosest first.
FP64_RTOL_CANDIDATES_3D = (1e-3, 1e-4, 1e-5, 1e-6)


def run_3d_fp64_plain(P, W, args, dev, barrier, job_rate, K3: int, refined_value: float) -> dict:
    """The 3D comparison of the refined path with plain FP64 at equal accuracy.
    From m0, `acc3d_steps` steps of the 3D workload on each leg: a plain FP64
    run at cg_rtol 1e-13 is the reference, and the relative L2 error of m is
    measured for the refined path (cg_rtol 1e-8) and for plain FP64 at each
    candidate tolerance.  The plain leg is then timed, like the refined one,
    over K3 steps after 3 warm-up steps at the loosest tolerance whose error
    is within ACC_BOUND."""
    import numpy as np
    import torch
    steps = args.acc3d_steps
    w = W.source_sink_3d(args.n3d)

    def make(precision, rtol):
        s = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                     cg_rtol=rtol, cg_maxit=5000, precond=PRECOND,
                     use_graph=not args.host_loop, device=str(dev))
        s.set_r(w.r)
        s.set_source(w.S)
        s.set_m(w.m0)
        return s

    def run(precision, rtol):
        with make(precision, rtol) as s:
            st = s.step(steps)
            return s.get_m(), st

    m_ref, st_ref = run("fp64", 1e-13)
    nref = float(np.linalg.norm(m_ref))
    legs = []
    for precision, rtol in [("fp32_refined", CG_RTOL_REFINED)] + \
            [("fp64", r) for r in FP64_RTOL_CANDIDATES_3D]:
        m, st = run(precision, rtol)
        legs.append({"precision": precision, "cg_rtol": rtol,
                     "m_rel_l2": float(np.linalg.norm(m - m_ref)) / nref,
                     "mean_cg_iters": st.total_cg_iters / steps})
    ok = [leg["cg_rtol"] for leg in legs[1:] if leg["m_rel_l2"] <= ACC_BOUND]
    rtol = max(ok) if ok else min(FP64_RTOL_CANDIDATES_3D)
    with make("fp64", rtol) as s:
        s.step(3)
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        st = s.step(K3)
        e1.record(s.stream)
        torch.cuda.synchronize()
    ms, v64 = job_rate(e0.elapsed_time(e1), w.npts * K3)
    return {"value": v64, "unit": UNIT, "ms_per_step": ms / K3, "steps": K3, "cg_rtol": rtol,
            "cg_iters_per_step": st.total_cg_iters / K3,
            "speedup_of_refined": refined_value / v64,
            "equal_accuracy": {"steps": steps, "bound": ACC_BOUND,
                               "reference": f"plain FP64 on the GPU, cg_rtol 1e-13, {steps} steps "
                                            f"from m0 ({st_ref.total_cg_iters / steps:.1f} CG "
                                            f"iterations per step)",
                               "legs": legs}}


# ----------------------------------------------------------------- equal accuracy
# Plain-FP64 tolerances tried for "equal accuracy", loosest first: the timed
# FP64 leg uses the loosest one whose m error after ACC_STEPS steps is within
# ACC_BOUND of the tight FP64 reference (calibrated: 1e-3 misses, 1e-4 meets).
FP64_RTOL_CANDIDATES = (1e-3, 1e-4, 1e-5)
ACC_STEPS = 100
ACC_BOUND = 1e-5


def equal_accuracy(P, W, dev, steps: int, legs, timed: bool = False) -> dict:
    """m after `steps` steps of the 2048^2 workload from m0, for each
    (precision, cg_rtol) leg, against a plain FP64 run at cg_rtol 1e-13 on the
    GPU: the relative L2 error of each leg (and, with timed, its throughput)."""
    import numpy as np
    import torch
    w = W.source_sink_2d(N_GRID, steps=steps)

    def run(precision, rtol):
        with P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision=precision,
                      cg_rtol=rtol, cg_maxit=5000, precond=PRECOND, device=str(dev)) as s:
            s.set_r(w.r)
            s.set_source(w.S)
            s.set_m(w.m0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = s.step(steps)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            return s.get_m(), st, secs

    m_ref, st_ref, _ = run("fp64", 1e-13)
    out = {"steps": steps, "bound": ACC_BOUND,
           "reference": f"plain FP64 on the GPU, cg_rtol 1e-13, {steps} steps from m0 "
                        f"({st_ref.total_cg_iters / steps:.1f} CG iterations per step)",
           "legs": []}
    nref = float(np.linalg.norm(m_ref))
    for precision, rtol in legs:
        m, st, secs = run(precision, rtol)
        leg = {"precision": precision, "cg_rtol": rtol,
               "m_rel_l2": float(np.linalg.norm(m - m_ref)) / nref,
               "mean_cg_iters": st.total_cg_iters / steps,
               "rel_residual_last_step": st.rel_residual}
        if timed:
            leg["mpoint_steps_per_s"] = w.npts * steps / secs / 1e6
        out["legs"].append(leg)
    return out


# ----------------------------------------------------------------- GB300 arm
def run_gb300(args) -> None:
    import numpy as np
    import torch
    import workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__._builder().build()
    if world > 1:
        torch.distributed.barrier()
    import paper_2606_06720_gb300 as P

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def reduce(x: float, op) -> float:
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=op)
        return float(t.item())

    def max_over_ranks(x: float) -> float:
        return x if world == 1 else reduce(x, torch.distributed.ReduceOp.MAX)

    def sum_over_ranks(x: float) -> float:
        return x if world == 1 else reduce(x, torch.distributed.ReduceOp.SUM)

    def job_rate(local_ms: float, local_units: float):
        """(slowest rank's ms, whole-job Mpoint-steps/s): the units every rank
        processed over the slowest rank's time (aggregate)."""
        ms, _, per_s = aggregate(local_ms, local_units, world, max_over_ranks, sum_over_ranks)
        return ms, per_s / 1e6

    # the FP64 residual kernels' roof, measured here (independent FMA chains on every SM)
    fp64_peak = P.fp64_fma_peak(reps=10)

    w = W.source_sink_2d(N_GRID)
    K, Wm = args.steps, args.warmup
    s = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp32_refined",
                 cg_rtol=CG_RTOL_REFINED, cg_maxit=2000, precond=PRECOND,
                 use_graph=not args.host_loop, sync_cert=args.sync_cert,
                 device=str(dev))
    s.set_r(w.r)
    s.set_source(w.S)
    s.set_m(w.m0)
    if args.inner_rtol:
        s.set_params(inner_rtol=args.inner_rtol)
    from paper_2606_06720_gb300.autotune import autotune
    s.step(1)  # realistic buffer contents for the tuner
    tune_report = {}
    tuning = autotune(s, reps=10, report=tune_report) if not args.no_tune else s.get_tuning()
    s.set_m(w.m0)
    s.set_p(np.zeros(w.shape))
    stream = s.stream
    if Wm > 0:
        s.step(Wm)
    torch.cuda.synchronize()

    # ---- timed region: K steps, device-resident inputs
    props = torch.cuda.get_device_properties(dev)
    gpu_id = ("GPU-" + str(props.uuid)) if getattr(props, "uuid", None) else str(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = s.launch_count()
    with ClockSampler(gpu_id, args.clocks_csv) as clk:
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        st = s.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier()
    launches = s.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    npts = w.npts
    ms_max, value = job_rate(ms, npts * K)
    iters_per_step = st.total_cg_iters / K
    sweeps_per_step = st.total_sweeps / K

    # ---- per-kernel durations (CUDA events around back-to-back launches, same data)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    res64 = st.total_refine_residuals / K  # FP64 residuals per step
    mid_per_step = st.total_mid_df / K     # double-float mid-step residuals per step
    counts = {"cg_grad": iters_per_step, "cg_apply": iters_per_step, "cg_div": iters_per_step,
              "cg_update": iters_per_step, "res_grad": res64, "res_apply": res64, "res_div": res64,
              "split_grad": 1, "split_row": 1, "split_heat": 1, "split_c2r": 1,
              "first_grad": 1, "first_apply": 1, "first_div": 1}
    if mid_per_step > 0:
        counts.update({"mid_grad": mid_per_step, "mid_apply": mid_per_step, "mid_div": mid_per_step})
    kernels = kernel_table(s, counts, BYTES_PER_POINT["fp32_refined"],
                           lambda k: fft_flops_per_point(k, *w.n), FP64_KERNELS["fp32_refined"],
                           npts, args.kernel_reps, hbm_peak, fp64_peak)
    bytes_step = sum(BYTES_PER_POINT["fp32_refined"][k] * npts * c for k, c in counts.items())
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    dk = kernels[dom]
    traffic = NCU_TRAFFIC_2048.get(dom) if w.n == (2048, 2048) else None
    if dk["bound"] == "alu":
        roofline = {"bound": "alu", "kernel": dom, "achieved": dk["alg_TFLOPs"],
                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": dk["frac"],
                    "traffic": traffic,
                    "peak_source": "measured: FP64 FMA throughput of this GPU in this run "
                                   "(hc_fp64_fma_peak: fastest of 10 launches; FMA = 2 flops); "
                                   "nominal 1.25",
                    "alg_bytes": BYTES_PER_POINT["fp32_refined"][dom] * npts}
    else:
        roofline = {"bound": "hbm", "kernel": dom, "achieved": dk["alg_GBs"], "peak": hbm_peak,
                    "unit": "GB/s", "frac": dk["frac"], "traffic": traffic,
                    "peak_source": hbm_src,
                    "alg_bytes": BYTES_PER_POINT["fp32_refined"][dom] * npts}
    share = dk["ms_per_step"] / (ms / K)
    roofline["share_of_step"] = share

    # ---- e2e through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Ke = max(5, K // 10)
        hm = torch.empty(2 * npts, dtype=torch.float64, pin_memory=True)
        hp = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        s.get_state(hm, hp)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            s.set_state(hm, hp)
            s.step(1)
            s.get_state(hm, hp)
        torch.cuda.synchronize()
        _, ve = job_rate((time.perf_counter() - t0) * 1e3, npts * Ke)
        barrier()
        e2e = {"value": ve, "unit": UNIT,
               "h2d_bytes_per_step": 3 * npts * 8, "d2h_bytes_per_step": 3 * npts * 8,
               "steps": Ke, "path": "hc_set_state (m, p from pinned host FP64) -> hc_step(1) -> "
                                    "hc_get_state (m, p to pinned host FP64)"}

    # ---- the same refined path with the refinement in double-float (FP32 pipes)
    dfv = None
    if not args.no_df:
        sdf = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt,
                       precision="fp32_refined_df", cg_rtol=CG_RTOL_REFINED, cg_maxit=2000,
                       precond=PRECOND, use_graph=not args.host_loop, device=str(dev))
        sdf.set_r(w.r)
        sdf.set_source(w.S)
        sdf.set_m(w.m0)
        sdf.step(1)
        if not args.no_tune:
            autotune(sdf, reps=10)
        sdf.set_m(w.m0)
        sdf.set_p(np.zeros(w.shape))
        sdf.step(Wm)
        Kd = max(10, K // 3)
        barrier()
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(sdf.stream)
        std = sdf.step(Kd)
        b1.record(sdf.stream)
        torch.cuda.synchronize()
        msd, vdf = job_rate(b0.elapsed_time(b1), npts * Kd)
        kdf = {}
        for name in ("res_grad", "res_apply", "res_div"):
            kms = sdf.time_kernel(name, reps=args.kernel_reps)
            kdf[name] = {"ms": kms,
                         "alg_TFLOPs": fft_flops_per_point(name, *w.n) * npts / (kms / 1e3) / 1e12,
                         "alg_GBs": BYTES_PER_POINT["fp32_refined"][name] * npts / (kms / 1e3) / 1e9}
        sdf.close()
        dfv = {"value": vdf, "unit": UNIT,
               "ms_per_step": msd / Kd, "steps": Kd,
               "cg_iters_per_step": std.total_cg_iters / Kd,
               "refine_sweeps_per_step": std.total_sweeps / Kd,
               "rel_residual_last_step": std.rel_residual,
               "refinement_arithmetic": "double-float (48-bit significand) on the FP32 pipes",
               "kernels": kdf}

    # ---- the headline path with the library's default preconditioner (reading
    # R3: kappa (-Laplacian), kappa = mean(r) + mean(|m|^2)/2): iteration counts
    # and throughput beside the anisotropic Kbar the timed legs use
    scal = None
    if not args.no_scalar:
        ss = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp32_refined",
                      cg_rtol=CG_RTOL_REFINED, cg_maxit=2000, precond="scalar",
                      use_graph=not args.host_loop, device=str(dev))
        ss.set_tuning(tuning["col_tile"], tuning["row_rows"], tuning["col_pipe"], tuning["row_pipe"])
        ss.set_r(w.r)
        ss.set_source(w.S)
        ss.set_m(w.m0)
        ss.step(Wm)
        Kc = K  # the headline's steps: iteration counts grow along the run
        barrier()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(ss.stream)
        stc = ss.step(Kc)
        c1.record(ss.stream)
        torch.cuda.synchronize()
        msc, vsc = job_rate(c0.elapsed_time(c1), npts * Kc)
        ss.close()
        scal = {"value": vsc, "unit": UNIT,
                "ms_per_step": msc / Kc, "steps": Kc, "precond": "scalar kappa (-Laplacian)",
                "cg_iters_per_step": stc.total_cg_iters / Kc,
                "rel_residual_last_step": stc.rel_residual}

    # ---- batched parameter sweep: 48 instances of mixed grids in one graph launch
    sweep = None
    if not args.no_sweep:
        mine = shard(48, rank, world)
        sws = [W.sweep_instance(i) for i in mine]
        solvers = []
        for wi in sws:
            si = P.Solver(wi.n, wi.L, c=wi.c, D=wi.D, gamma=wi.gamma, dt=wi.dt,
                          precision="fp32_refined", cg_rtol=CG_RTOL_REFINED, cg_maxit=2000,
                          precond=PRECOND, device=str(dev))
            si.set_r(wi.r)
            si.set_source(wi.S)
            si.set_m(wi.m0)
            solvers.append(si)
        if not args.no_tune:
            done_sizes = set()
            for si in solvers:  # one tuning per grid size (the cache serves the rest)
                if si.n not in done_sizes:
                    si.step(1)
                    autotune(si, reps=5)
                    si.set_m(sws[solvers.index(si)].m0)
                    si.set_p(np.zeros(si.shape))
                    done_sizes.add(si.n)
            for si in solvers:
                autotune(si, reps=5)
        batch = P.Batch(solvers, stream=stream)
        ncls, nbat = batch.classes()
        batch.step(3)
        Ks = max(20, K // 15)  # a 20-step window at least of the 1000-step sweep
        barrier()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        sts = batch.step(Ks)
        c1.record(stream)
        torch.cuda.synchronize()
        pts = sum(wi.npts for wi in sws)  # this rank's shard
        mss, vsw = job_rate(c0.elapsed_time(c1), pts * Ks)
        batch.close()
        for si in solvers:
            si.close()
        sweep = {"value": vsw, "unit": UNIT,
                 "ms_per_step": mss / Ks, "steps": Ks, "instances": 48,
                 "instances_per_rank": len(sws),
                 "workload": "48 instances: 16x128^2, 16x256^2, 16x512^2; (c,D,gamma) over "
                             "{5,10,25,50}x{0.01,0.02,0.05,0.1}x{0.5,0.75,1}; r=0.1, centred "
                             "Gaussian S, m0~U[0,1] seed i, dt=1e-3, FP32 + FP64 refinement",
                 "cg_iters_per_step_mean": sum(x.total_cg_iters for x in sts) / Ks / len(sts),
                 "max_rel_residual": max(x.rel_residual for x in sts),
                 "one_graph_launch_per_step": True,
                 "size_classes": ncls, "batched_instances": nbat,
                 "launch_structure": "one graph launch per step; inside it, one kernel launch "
                                     "per pass of the step per size class over all its "
                                     "instances (blockIdx.y = instance)"}

    # ---- adjoint: loss ||m(T) - m_target||^2 on the 1024^2 problem, checkpointed
    adjv = None
    if not args.no_adjoint:
        wa = W.source_sink_2d(1024, gamma=0.75)
        wt = W.source_sink_2d(1024, gamma=0.75, seed=1)
        Ka, every = args.adj_steps, max(1, min(args.adj_every, args.adj_steps))
        sa = P.Solver(wa.n, wa.L, c=wa.c, D=wa.D, gamma=wa.gamma, dt=wa.dt,
                      precision="fp32_refined", cg_rtol=CG_RTOL_REFINED, cg_maxit=2000,
                      precond=PRECOND, device=str(dev))
        sa.set_r(wa.r)
        sa.set_source(wa.S)
        if not args.no_tune:
            sa.set_m(wa.m0)
            sa.step(1)
            autotune(sa, reps=5)
        sa.set_m(wt.m0)
        sa.set_p(np.zeros(wa.shape))
        sa.step(Ka)
        m_target = sa.get_m()
        sa.set_m(wa.m0)
        sa.set_p(np.zeros(wa.shape))
        sa.step(Ka)
        lamT = 2.0 * (sa.get_m() - m_target)
        sa.set_m(wa.m0)
        sa.set_p(np.zeros(wa.shape))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grads = sa.adjoint(Ka, lamT, every=every)
        torch.cuda.synchronize()
        msa, vadj = job_rate((time.perf_counter() - t0) * 1e3, wa.npts * Ka)
        sa.close()
        adjv = {"value": vadj, "unit": UNIT,
                "ms_per_step": msa / Ka, "steps": Ka, "checkpoint_every": every,
                "workload": "1024x1024 source/sink, gamma=0.75, c=25, D=0.02, dt=5e-4, FP32 + FP64 "
                            "refinement; loss ||m(T) - m_target||^2, m_target from a forward run "
                            "from the seed-1 m0; the time covers the checkpointed forward, the "
                            "segment recomputation and the reverse sweep (gradients for c^2, D^2, "
                            "r, S, m0)",
                "dL_dc2": grads["dc2"], "dL_dD2": grads["dD2"]}

    # ---- diagnostics (Section 2.5) and Algorithm 1's loop with its stopping rules
    diag = None
    if not args.no_diag:
        diag = run_diagnostics(P, W, args, dev, barrier, job_rate, value)

    # ---- the paper's grid-convergence setup on its N = 50 2^k grids (mixed radix)
    conv = None
    if not args.no_conv:
        conv = run_convergence(P, W, args, dev, job_rate)

    # ---- 3D: the 256^3 source/sink problem (d = 3), FP32 + FP64 refinement
    three_d = None
    if not args.no_3d:
        three_d = run_3d(P, W, args, dev, barrier, job_rate, hbm_peak, hbm_src, fp64_peak)

    # ---- equal accuracy (every rank runs its own replica): the refined path
    # and the plain FP64 path at each candidate tolerance, 100 steps from m0,
    # against a plain FP64 run at cg_rtol 1e-13
    acc = None
    fp64_rtol = FP64_EQUAL_RTOL
    if not args.no_fp64:
        acc = equal_accuracy(P, W, dev, ACC_STEPS,
                             [("fp32_refined", CG_RTOL_REFINED)] +
                             [("fp64", r) for r in FP64_RTOL_CANDIDATES])
        ok = [leg["cg_rtol"] for leg in acc["legs"][1:] if leg["m_rel_l2"] <= ACC_BOUND]
        fp64_rtol = max(ok) if ok else min(FP64_RTOL_CANDIDATES)

    # ---- plain FP64 path at equal accuracy
    fp64 = None
    if not args.no_fp64:
        K64 = max(3, K // 20)
        s64 = P.Solver(w.n, w.L, c=w.c, D=w.D, gamma=w.gamma, dt=w.dt, precision="fp64",
                       cg_rtol=fp64_rtol, cg_maxit=5000, precond=PRECOND,
                       use_graph=True, device=str(dev))
        s64.set_r(w.r)
        s64.set_source(w.S)
        s64.set_m(w.m0)
        s64.step(1)
        if not args.no_tune:
            autotune(s64, reps=3)
        s64.set_m(w.m0)
        s64.set_p(np.zeros(w.shape))
        s64.step(max(Wm, 3))
        barrier()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s64.stream)
        st64 = s64.step(K64)
        a1.record(s64.stream)
        torch.cuda.synchronize()
        ms64, v64 = job_rate(a0.elapsed_time(a1), npts * K64)
        k64 = {}
        for name in ("cg_apply", "cg_div", "cg_grad"):
            kms = s64.time_kernel(name, reps=max(3, args.kernel_reps // 5))
            tfl = fft_flops_per_point(name, *w.n) * npts / (kms / 1e3) / 1e12
            k64[name] = {"ms": kms, "alg_TFLOPs": tfl, "frac_of_fp64_peak": tfl / fp64_peak}
        s64.close()
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / K64, "steps": K64,
                "cg_rtol": fp64_rtol, "cg_iters_per_step": st64.total_cg_iters / K64,
                "kernels": k64, "speedup_of_refined": value / v64}

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        secs, threads, it = oracle_steps(N_GRID, 1, warm=1)
        cpu = {"value": npts / secs / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"one warm-started FP64 oracle step of the same 2048x2048 workload "
                         f"(after one untimed step), cg_rtol {CG_RTOL_REFINED}, {it} CG iterations"}

    closed_inner = s.params.inner_rtol
    s.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"tuning": tuning, "inner_rtol": closed_inner,
                                       "tuning_us": tune_report.get("us")}),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "fp64_fma_peak_tflops": fp64_peak,
            "hbm_gbs": bytes_step * K / (ms / 1e3) / 1e9,
            "cg_iters_per_step": iters_per_step, "refine_sweeps_per_step": sweeps_per_step,
            "fp64_residuals_per_step": res64, "df_mid_residuals_per_step": mid_per_step,
            "cg_iterations_per_s": sum_over_ranks(iters_per_step * K) / (ms_max / 1e3),
            "rel_residual_last_step": st.rel_residual,
            "m_rel_l2_refined": acc["legs"][0]["m_rel_l2"] if acc else None,
            "m_rel_l2_fp64_plain": next((leg["m_rel_l2"] for leg in acc["legs"][1:]
                                         if leg["cg_rtol"] == fp64_rtol), None) if acc else None,
            "fp64_plain_value": fp64["value"] if fp64 else None,
            "speedup_vs_fp64_plain": fp64["speedup_of_refined"] if fp64 else None,
            "equal_accuracy": acc,
            "fp64_plain": fp64, "refined_df": dfv, "scalar_kappa": scal, "sweep": sweep,
            "adjoint": adjv,
            "three_d": three_d, "diagnostics": diag, "paper_convergence": conv,
            "kernels": kernels,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_only_3d(args) -> None:
    import torch
    import workloads as W
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2606_06720_gb300 as P
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_FALLBACK)
    out = run_3d(P, W, args, torch.device("cuda", 0), lambda: None,
                 lambda ms, units: (ms, units / (ms / 1e3) / 1e6), hbm_peak,
                 "measured" if "hbm_gbs" in peaks else "fallback", P.fp64_fma_peak(reps=5))
    print(json.dumps(out), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--ref-n", type=int, default=0,
                    help="reference arm: oracle sample grid (0: 2048 up to 20 steps, 1024 up to "
                         "80, else 512)")
    ap.add_argument("--kernel-reps", type=int, default=30)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-df", action="store_true", help="skip the double-float refinement leg")
    ap.add_argument("--no-scalar", action="store_true",
                    help="skip the leg with the default scalar-kappa preconditioner")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched 48-instance sweep leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--adj-steps", type=int, default=500, help="adjoint leg: steps")
    ap.add_argument("--adj-every", type=int, default=50, help="adjoint leg: checkpoint spacing")
    ap.add_argument("--no-3d", action="store_true", help="skip the 3D (256^3) leg")
    ap.add_argument("--no-diag", action="store_true",
                    help="skip the diagnostics / stopping-rule leg")
    ap.add_argument("--n3d", type=int, default=256, help="3D leg: grid points per axis")
    ap.add_argument("--acc3d-steps", type=int, default=5,
                    help="3D leg: steps from m0 of the equal-accuracy comparison with plain FP64")
    ap.add_argument("--no-conv", action="store_true",
                    help="skip the paper's grid-convergence leg (N = 50 .. 800, mixed radix)")
    ap.add_argument("--conv-steps", type=int, default=100,
                    help="convergence leg: steps (100 reach the paper's t = 5)")
    ap.add_argument("--only-3d", action="store_true",
                    help="run only the 3D leg, --steps/--warmup steps (for profiling)")
    ap.add_argument("--inner-rtol", type=float, default=0.0,
                    help="inner FP32 CG reduction factor (0: library default)")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--sync-cert", action="store_true",
                    help="headline leg: certify each step before the next (hc_params.sync_cert)")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven CG loop instead of graphs (ncu cannot profile kernel "
                         "nodes of graphs with conditional nodes)")
    ap.add_argument("--accuracy", action="store_true", help="equal-accuracy calibration")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the raw nvidia-smi samples of the timed region in this file")
    ap.add_argument("--acc-steps", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        run_reference(args)
    elif args.only_3d:
        run_only_3d(args)
    elif args.accuracy:
        run_accuracy(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
