"""Benchmark of one time step of the vorticity--stream-vector phase-field
method (phi update, mu, source, six Poisson solves) on GB300.

Default: N = 1 GPU, the Couette vesicle at 512 x 256 x 256 (x flow axis,
256 x 256 cross-section, the 256^2 x 512 workload), mixed precision (FP32
storage and smoothing, exact FP64-class defect, FP64 reductions), beside the
plain-FP64 step with the same multigrid schedule.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank advances its own replica (the method has no
exchange step on one GPU per problem); value = all ranks' cell-steps / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
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

import numpy as np  # noqa: E402

METRIC = "Mcell-steps/s at 256^2x512 (mixed FP32/FP64-defect; plain FP64 beside it)"
UNIT = "Mcell-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--nz", type=int, default=256)
    ap.add_argument("--cycles", type=int, default=None,
                    help="V-cycles per Poisson solve (default: BENCH_CYCLES)")
    ap.add_argument("--extrapolate", type=int, default=None, choices=[0, 1, 2],
                    help="order of the first guess of each solve from the previous solutions "
                         "(default: BENCH_EXTRAPOLATE)")
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the 512x256x256 line: N independent seeded problems of "
                         "a parameter sweep stepped together (batched CUDA graph)")
    ap.add_argument("--poisson-case", action="store_true",
                    help="instead of the benchmark: one single-component mixed Poisson solve "
                         "(2 V-cycles, seeded rhs) on the nx x ny x nz grid, for kernel profiles")
    return ap.parse_args()


def run_poisson_case(args):
    """A small, fixed launch sequence for ncu captures of the solver kernels:
    every multigrid kernel of the mixed path at the benchmark's plane size,
    with a single component (fields of nx*ny*nz*4 bytes, 134 MB at the
    default size: above L2, a few GB on the device in all)."""
    import inputs
    from paper_2601_05031_gb300 import build
    build.build()
    from paper_2601_05031_gb300 import vsv as V
    from paper_2601_05031_gb300.sim import Simulation
    b = inputs.random_field((args.nz, args.ny, args.nx), seed=3)
    sim = Simulation(args.nx, args.ny, args.nz, 1.0, V.VSV_MIXED)
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, True), tol=0.0, max_cycles=2,
                                       check=False)
    sim.close()
    print(json.dumps({"poisson_case": [args.nx, args.ny, args.nz], "cycles": cyc,
                      "rel_residual": rr}), flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(REASONS, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- replicas
def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the slowest replica's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, cells_per_rank, steps, ms_max):
    """Whole-job Mcell-steps/s: every rank's cell-steps over the slowest time."""
    return world_size * cells_per_rank * steps / (ms_max * 1e-3) / 1e6


# ---------------------------------------------------------------- GPU arm
GUESS = {0: "previous solution x^n", 1: "extrapolated guess 2x^n - x^(n-1)",
         2: "extrapolated guess 3x^n - 3x^(n-1) + x^(n-2)"}

# DRAM traffic of the finest-level fused sweeps per cell and component:
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of each
# variant (zero-input 6.86, plain 11.78, update 23.45 B per cell) on a
# single-component 512 x 256 x 256 solve, weighted 1:2:1 as a V(2,2)-cycle
# launches them.  It belongs to the kernel sources whose digest is
# FUSED_SWEEP_TRAFFIC_BUILD; with any other sources the line reports null.
FUSED_SWEEP_TRAFFIC_PER_CELL = 13.47
FUSED_SWEEP_TRAFFIC_BUILD = "aaa3109bbdbfb5e1"
FUSED_SWEEP_SOURCES = ("paper_2601_05031_gb300/csrc/smooth.cu", "paper_2601_05031_gb300/csrc/tile.cuh",
                       "paper_2601_05031_gb300/csrc/common.cuh", "paper_2601_05031_gb300/csrc/internal.h")


def fused_sweep_build():
    """Digest of the fused sweep's kernel sources (first 16 hex digits of
    their SHA-256)."""
    h = hashlib.sha256()
    for f in FUSED_SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]

# steps per captured graph (the library's replay length)
GRAPH_STEPS = 6

# The benchmark's solver schedule: fixed V(2,2)-cycles per Poisson solve
# from the first guess extrapolated in time (order BENCH_EXTRAPOLATE from
# the previous solutions), with the library's default over-relaxed
# red-black smoothing (omega_mg 1.3).  The long-run tests check this
# schedule against FP64 solved to 1e-12 every step.
BENCH_CYCLES = 2
BENCH_EXTRAPOLATE = 2


def make_sim(w, prec, cycles, extrapolate=1, stream=None):
    from paper_2601_05031_gb300 import vsv as V
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, prec, stream=stream)
    sp = sim.solver_params()
    sp.fixed_cycles = cycles
    sp.extrapolate = extrapolate
    sp.tol = 1e-7 if prec == V.VSV_MIXED else 1e-12
    V.vsv_set_solver(sim.g, sp)
    sim.set_phi(w.phi0)
    return sim


def timed_steps(sim, nsteps, dt, torch, barrier, stepper=None):
    """Device time of `nsteps` steps by events on the grid's stream: one
    vsv_step call, or with `stepper` (a one-grid Batch) the graph replays.
    The batch's stream waits for the grid's queued work (the start event)
    before its replays, and the grid's stream waits for the replays before
    any leftover single steps, so the grid's stream brackets all of it."""
    st = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    if stepper is None:
        sim.step(nsteps, dt)
    else:
        stepper.step(nsteps, dt)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1)


def field_errors(sa, sb, V, torch):
    """Relative L2 error of every field of sa against sb: phi, mu, and the
    vector fields omega, psi (full, base flow included) and velocity, each
    over its three components and per component."""
    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    def get(s, fid):
        return s.field(fid, np.float64, on_device=True)
    errs = {"phi": rel(get(sa, V.VSV_FIELD_PHI), get(sb, V.VSV_FIELD_PHI)),
            "mu": rel(get(sa, V.VSV_FIELD_MU), get(sb, V.VSV_FIELD_MU))}
    for name, f0 in (("omega", V.VSV_FIELD_OMEGA_X), ("psi", V.VSV_FIELD_PSI_X),
                     ("vel", V.VSV_FIELD_VEL_X)):
        num = den = 0.0
        for c in range(3):
            a, b = get(sa, f0 + c), get(sb, f0 + c)
            d2, n2 = float(torch.linalg.vector_norm(a - b)) ** 2, float(torch.linalg.vector_norm(b)) ** 2
            errs[f"{name}_{'xyz'[c]}"] = (d2 / n2) ** 0.5 if n2 > 0 else d2 ** 0.5
            num, den = num + d2, den + n2
        errs[name] = (num / den) ** 0.5
    return errs


def run_gpu(args, ws, rank, local):
    import torch
    import inputs
    from paper_2601_05031_gb300 import build as B
    from paper_2601_05031_gb300 import vsv as V

    if rank == 0 or not B.up_to_date():
        B.build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    w = inputs.vesicle_couette_512x256x256(nx=args.nx, ny=args.ny, nz=args.nz)
    N = w.ncells
    from paper_2601_05031_gb300.sim import Batch
    # the grid on a stream of its own, stepped through a one-grid batch: the
    # library captures six steps (the period of its buffer rotation) into a
    # CUDA graph once and replays it, leftover steps one call each
    sim = make_sim(w, V.VSV_MIXED, args.cycles, args.extrapolate, stream=torch.cuda.Stream())
    batch = Batch([sim])
    for _ in range(args.warmup):
        sim.step(1, w.dt)
    batch.step(GRAPH_STEPS, w.dt)      # capture and one replay, untimed
    warmup = args.warmup + GRAPH_STEPS
    torch.cuda.synchronize()
    launches0, bytes0 = sim.kernel_launches(), sim.kernel_bytes()
    with ClockSampler(local) as clk:
        ms_local = timed_steps(sim, args.steps, w.dt, torch, barrier, stepper=batch)
    launches = sim.kernel_launches() - launches0
    step_bytes = (sim.kernel_bytes() - bytes0) / args.steps
    batch.close()
    # the same steps without the graph, one vsv_step call, for comparison
    ms_nograph = timed_steps(sim, args.steps, w.dt, torch, barrier)
    ms_nograph = max_over_ranks(ms_nograph, dist, "cuda")
    ms = ms_local
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(ws, N, args.steps, ms)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded prolate vesicle, V_r 0.9, eps 1.5, Couette +-0.05)",
        "config": {"workload": w.name, "grid_xyz": [w.nx, w.ny, w.nz], "cells": N,
                   "precision": "mixed: f32 fields and smoothing, exact (FP64-class) defect, "
                                "f64 reductions",
                   "solver": f"multigrid V(2,2), red-black SOR smoothing (omega 1.3), "
                             f"{args.cycles} cycles per Poisson solve from the "
                             f"{GUESS[args.extrapolate]}, 6 solves per step",
                   "l2": "inputs larger than L2 (about 2 GB of resident fields per replica)",
                   "dt": w.dt, "parallelism": f"replicas x{ws}",
                   "launch": f"CUDA graph of {GRAPH_STEPS} steps captured by the library "
                             "(vsv_batch_step on one grid), replayed"},
        "gpu_launches": int(launches),
        "without_graph": {"value": round(job_throughput(ws, N, args.steps, ms_nograph), 3),
                          "unit": UNIT, "ms_per_step": round(ms_nograph / args.steps, 4),
                          "launch": "one vsv_step call for all steps"},
    }
    # whole-step HBM rate in the algorithmic sense: the bytes every kernel of
    # a step must move (tallied by the library per launch) over the step time
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    step_gbs = step_bytes / (ms_local / args.steps * 1e-3) / 1e9
    out["hbm_step"] = {"algorithmic_bytes_per_step": round(step_bytes),
                       "bytes_per_cell_step": round(step_bytes / N, 1),
                       "achieved_gbs": round(step_gbs, 1), "unit": "GB/s",
                       "frac_of_measured": round(step_gbs / peak, 4),
                       "frac_of_nominal_8tbs": round(step_gbs / 8000.0, 4)}
    # roofline of the dominant kernel: fine-level red-black half-sweeps, timed
    # live with events on the library's stream during extra timed steps
    V.vsv_profile_enable(sim.g, V.VSV_KCLASS_SMOOTH_FINE)
    nprof = max(2, min(args.steps, 5))
    timed_steps(sim, nprof, w.dt, torch, barrier)
    pms, pn, pbytes = V.vsv_profile_read(sim.g, V.VSV_KCLASS_SMOOTH_FINE, with_bytes=True)
    V.vsv_profile_enable(sim.g, V.VSV_KCLASS_SMOOTH_FINE, False)
    build = fused_sweep_build()
    traffic_ok = build == FUSED_SWEEP_TRAFFIC_BUILD
    per_launch_s = pms * 1e-3 / max(pn, 1)
    algo = pbytes / max(pn, 1)
    achieved = algo / per_launch_s / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "k_rbgs_fused (finest level: one full red-black "
                       "sweep of 3 components; 12 B/cell, 8 with zero input, 24 when it also "
                       "updates the double-word iterate)", "achieved": round(achieved, 1),
                       "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                       "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                       "algorithmic_bytes_per_launch": round(algo), "launches_timed": int(pn),
                       "avg_launch_us": round(per_launch_s * 1e6, 2),
                       "traffic": (round(FUSED_SWEEP_TRAFFIC_PER_CELL * N * 3) if traffic_ok
                                   else None),
                       "traffic_source": ("ncu capture of this kernel build (profiles/"
                                          "fused_sweep_poisson_512x256x256.md), per cell "
                                          "and component x cells x 3" if traffic_ok else
                                          "no ncu capture of this kernel build"),
                       "kernel_build": build}
    out["clocks"] = clk.summary()
    # plain FP64 step with the same schedule, and the accuracy of mixed vs FP64
    if not args.no_fp64:
        k64 = args.fp64_steps or max(3, args.steps // 4)
        sim64 = make_sim(w, V.VSV_FP64, args.cycles, args.extrapolate)
        for _ in range(min(args.warmup, 3)):
            sim64.step(1, w.dt)
        ms64 = timed_steps(sim64, k64, w.dt, torch, barrier)
        v64 = N * k64 / (ms64 * 1e-3) / 1e6
        # accuracy: the benchmarked mixed schedule against FP64 solved to a
        # relative residual of 1e-12 every step, same phi0 and steps
        nacc = 10
        simA = make_sim(w, V.VSV_MIXED, args.cycles, args.extrapolate)
        simB = make_sim(w, V.VSV_FP64, 0)
        simA.step(nacc, w.dt)
        simB.step(nacc, w.dt)
        errs = field_errors(simA, simB, V, torch)
        simA.close(); simB.close()
        out["fp64"] = {"value": round(v64, 3), "unit": UNIT, "ms_per_step": round(ms64 / k64, 3),
                       "steps": k64, "speedup_mixed_over_fp64": round(value / (ws * v64), 3),
                       "kernels": "per-colour reference sweeps and level-by-level transfers in "
                                  "FP64 (FP64-ALU-bound on GB300), not the fused FP32 sweeps"}
        out["accuracy_mixed_vs_fp64"] = {"steps": nacc, "reference": "FP64 path, every solve to "
                                         "relative residual 1e-12", "rel_l2": errs}
        sim64.close()
    # end to end through the C ABI with host buffers: phi in from pinned host
    # memory, one step, phi out to pinned host memory, every step.  phi goes
    # both ways in FP64, which carries the double-word state exactly.  The
    # headline uses the asynchronous transfers (VSV_HOST_ASYNC: copy-engine
    # streams of the grid overlap the copies with the steps; one vsv_check at
    # the end, inside the timed region, makes the last output valid); the
    # synchronous calls are timed beside it.
    if not args.no_e2e:
        host_in = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float64, pin_memory=True)
        host_out = torch.empty((w.nz, w.ny, w.nx), dtype=torch.float64, pin_memory=True)
        host_in.copy_(sim.field(V.VSV_FIELD_PHI, np.float64, on_device=True).cpu())
        ke = max(2, min(args.steps, 5))

        def e2e_run(kind):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(ke):
                V.vsv_set_field(sim.g, V.VSV_FIELD_PHI, host_in.data_ptr(), V.VSV_DTYPE_F64, kind)
                sim.step(1, w.dt)
                V.vsv_get_field(sim.g, V.VSV_FIELD_PHI, host_out.data_ptr(), V.VSV_DTYPE_F64, kind)
            V.vsv_check(sim.g)
            te = time.perf_counter() - t0
            return max_over_ranks(te * 1e3, dist, "cuda") * 1e-3

        e2e_run(V.VSV_HOST_ASYNC)            # warm-up of the copy streams
        ta = e2e_run(V.VSV_HOST_ASYNC)
        tsync = e2e_run(0)
        out["e2e"] = {"value": round(ws * N * ke / ta / 1e6, 3), "unit": UNIT,
                      "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8, "steps": ke,
                      "transfers": "asynchronous (VSV_HOST_ASYNC): copy-engine streams overlap "
                                   "the copies with the steps",
                      "synchronous": round(ws * N * ke / tsync / 1e6, 3)}
    sim.close()
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU oracle
def oracle_sample_workload(nsteps_hint=3):
    """The same recipe (Couette, V_r 0.9, eps 1.5, seeded axes scaled to the
    cross-section) at 256 x 128 x 128: 1/8 of the benchmark's cells."""
    import inputs
    return inputs.vesicle_couette_512x256x256(nx=256, ny=128, nz=128, nsteps=nsteps_hint)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def time_oracle(steps, workers):
    """Wall time of `steps` oracle steps of the sample workload, its FFT and
    DST primitives run with `workers` threads (the oracle itself unchanged;
    the element-wise numpy work stays on one thread)."""
    import scipy.fft
    import oracle
    ws = oracle_sample_workload(steps)
    p = oracle.params_from_workload(ws)
    with scipy.fft.set_workers(workers):
        st = oracle.init_state(p, ws.phi0)
        t0 = time.perf_counter()
        for _ in range(steps):
            oracle.step(st, ws.dt)
        t = time.perf_counter() - t0
    return ws, t


def cpu_baseline(w_full, steps=2):
    """The oracle on the host cores: one thread, and every core for its FFT /
    DST work.  Reported in Mcell-steps/s of the sampled grid."""
    ncores = os.cpu_count() or 1
    ws, t1 = time_oracle(steps, 1)
    _, tn = time_oracle(steps, ncores)
    v1 = ws.ncells * steps / t1 / 1e6
    vn = ws.ncells * steps / tn / 1e6
    frac = w_full.ncells // ws.ncells
    return {"value": round(vn, 4), "unit": UNIT, "cores": ncores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": ncores,
            "one_thread": {"value": round(v1, 4), "unit": UNIT, "cores": 1},
            "sample": f"{steps} oracle steps of the same recipe at {ws.nx}x{ws.ny}x{ws.nz} "
                      f"(1/{frac} of the cells; per-cell rate, extrapolated to the full grid), "
                      f"exact DST/FFT Poisson solves in numpy/scipy FP64; 'value' with the "
                      f"FFT/DST primitives on all {ncores} cores, 'one_thread' on one"}


def run_batch(args, ws, rank, local):
    """N independent problems (sizes 32-192 x 32-96 x 32-96, droplets and
    vesicles, Ca log-uniform 0.05-5) stepped as one batch: a captured CUDA
    graph of six steps of all of them, each on its own stream.  Beside it,
    the same problems stepped one call per grid (streams, no graph)."""
    import torch
    import inputs
    from paper_2601_05031_gb300 import build as B
    from paper_2601_05031_gb300 import vsv as V
    from paper_2601_05031_gb300.sim import Simulation, Batch
    if not B.up_to_date():
        B.build()
    torch.cuda.set_device(local)
    wl = inputs.batch_instances(n=args.batch, seed=rank)
    cells = sum(w.ncells for w in wl)
    dt = wl[0].dt

    def make():
        sims = []
        for w in wl:
            s = Simulation.from_workload(w, V.VSV_MIXED, stream=torch.cuda.Stream())
            sp = s.solver_params()
            sp.fixed_cycles = args.cycles
            sp.extrapolate = args.extrapolate
            V.vsv_set_solver(s.g, sp)
            s.set_phi(w.phi0)
            sims.append(s)
        return sims

    steps = max(6, (args.steps // 6) * 6)
    sims = make()
    batch = Batch(sims)
    batch.step(max(args.warmup, 2) + 6, dt)        # warm-up, history, capture
    torch.cuda.synchronize()
    launches0 = sum(s.kernel_launches() for s in sims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(batch.stream)
        batch.step(steps, dt)
        e1.record(batch.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = sum(s.kernel_launches() for s in sims) - launches0
    batch.close()
    # the same work without the graph: one vsv_step call per grid and step
    for s in sims:
        s.step(2, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for s in sims:
            s.step(1, dt, check=False)
    torch.cuda.synchronize()
    ms_plain = (time.perf_counter() - t0) * 1e3
    for s in sims:
        s.close()
    value = cells * steps / (ms * 1e-3) / 1e6
    out = {"metric": "Mcell-steps/s (batch of independent problems)", "value": round(value, 3),
           "unit": "Mcell-steps/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
           "ms_per_step": round(ms / steps, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded parameter sweep)",
           "config": {"workload": f"batch_{args.batch}_instances", "instances": args.batch,
                      "cells": cells, "solver": f"{args.cycles} V(2,2)-cycles per solve",
                      "launch": "one captured CUDA graph of 6 steps of every instance"},
           "gpu_launches": int(launches), "clocks": clk.summary(),
           "without_graph": {"value": round(cells * steps / (ms_plain * 1e-3) / 1e6, 3),
                             "unit": "Mcell-steps/s",
                             "launch": "one vsv_step call per instance and step"}}
    print(json.dumps(out), flush=True)


def run_reference(args, ws, rank):
    """The oracle as it stands on the host cores (its FFT / DST primitives on
    every core), each step one oracle step of the sampled workload."""
    if rank != 0:
        return
    import inputs
    import scipy.fft
    import oracle
    w_full = inputs.vesicle_couette_512x256x256(nx=args.nx, ny=args.ny, nz=args.nz)
    ncores = os.cpu_count() or 1
    ws_ = oracle_sample_workload()
    p = oracle.params_from_workload(ws_)
    with scipy.fft.set_workers(ncores):
        st = oracle.init_state(p, ws_.phi0)
        for _ in range(args.warmup):
            oracle.step(st, ws_.dt)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.step(st, ws_.dt)
        t = time.perf_counter() - t0
    value = ws_.ncells * args.steps / t / 1e6
    sample = (f"each step one oracle step of the same recipe at {ws_.nx}x{ws_.ny}x{ws_.nz} "
              f"(1/{w_full.ncells // ws_.ncells} of the cells; per-cell rate), numpy/scipy "
              f"FP64, FFT/DST primitives on {ncores} cores")
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(t / args.steps * 1e3, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w_full.name, "grid_xyz": [w_full.nx, w_full.ny, w_full.nz],
                      "sampled_grid_xyz": [ws_.nx, ws_.ny, ws_.nz]},
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": ncores,
                            "kind": "oracle", "cpu_model": cpu_model(), "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.cycles is None:
        args.cycles = BENCH_CYCLES
    if args.extrapolate is None:
        args.extrapolate = BENCH_EXTRAPOLATE
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.poisson_case:
        if rank == 0:
            run_poisson_case(args)
        return
    if args.batch > 0:
        run_batch(args, ws, rank, local)
        return
    run_gpu(args, ws, rank, local)


if __name__ == "__main__":
    main()
