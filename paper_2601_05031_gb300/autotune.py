"""Schedule autotuner for the mixed path: per size class, the cheapest fixed
multigrid schedule (V-cycles per solve, order of the first guess in time)
whose velocity stays within a target of the converged answer, the faster
tiling mode for it (solver variant 0: fused and tiled kernels with partial
edge tiles; variant 2: those kernels on tile-aligned levels only, per-colour
and row kernels elsewhere), and the fastest launch shape (the components'
solves on one stream or on a stream each, programmatic dependent launches
on or off, the levels below the finest level by level or as one cooperative
launch).

A fixed schedule (``fixed_cycles`` > 0) is what batched stepping and the
benchmark use: no host synchronisation inside a step.  How many cycles it
needs depends on the grid (multigrid depth, coarsest level), the flow and the
body, so it is measured rather than guessed: each candidate runs a few steps
from the workload's initial state and is compared with the same steps solved
to a relative residual of ``ref_tol`` (FP64-class on the mixed path).  The
cheapest candidate by measured step time that stays below ``target / margin``
wins.  The tiling modes and launch shapes give bit-identical results, so
they are compared by time alone, on the winning schedule (plain stepping:
each candidate's step time over one vsv_step call, the grid alone on the
GPU).  Many small grids stepped side by side favour other shapes than one
grid alone (the library's size-based defaults); pass ``shapes=()`` to keep
those for a batch.  Results are cached per size class (flow, free energy, and the powers of
two nearest to the extents), so a batch of many problems tunes each class
once.

Everything runs through the C ABI (vsv_*); no arithmetic of the method
happens here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import vsv as V
from .sim import Simulation

DEFAULT_CANDIDATES = ((2, 2), (3, 1), (3, 2), (4, 1), (4, 2), (5, 1), (6, 1))
# launch shapes (component_streams, launch_overlap, lower_cycle); the
# component streams are off with the cooperative lower cycle
DEFAULT_SHAPES = ((0, 0, 0), (0, 1, 0), (1, 0, 0), (1, 1, 0), (0, 1, 1))


@dataclass
class TunedSchedule:
    fixed_cycles: int
    extrapolate: int
    ms_per_step: float
    vel_err: float
    trials: list
    variant: int = 0          # tiling mode (solver variant 0 or 2)
    tiling_ms: dict = None    # ms per step of the winning schedule per tiling mode
    shape: tuple = (2, 2, 0)  # (component_streams, launch_overlap, lower_cycle)
    shape_ms: dict = None     # ms per step of the winning schedule and mode per shape


_CACHE: dict = {}


def size_class(w) -> tuple:
    """Flow kind, free energy and the nearest powers of two of the extents."""
    p2 = lambda n: int(round(math.log2(max(n, 1))))
    return (w.flow_kind, w.fe_kind, p2(w.nx), p2(w.ny), p2(w.nz))


def _velocity(sim):
    return torch.stack([sim.field(V.VSV_FIELD_VEL_X + c, np.float64, on_device=True)
                        for c in range(3)])


def _run(w, steps, solver_setup):
    sim = Simulation.from_workload(w, V.VSV_MIXED, stream=torch.cuda.Stream())
    sp = sim.solver_params()
    solver_setup(sp)
    V.vsv_set_solver(sim.g, sp)
    sim.set_phi(w.phi0)
    st = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    sim.step(steps, w.dt)
    e1.record(st)
    torch.cuda.synchronize()
    vel = _velocity(sim)
    sim.close()
    return vel, e0.elapsed_time(e1) / steps


def tune(w, target=1e-6, margin=3.0, steps=6, candidates=DEFAULT_CANDIDATES, ref_tol=1e-11,
         use_cache=True, tilings=(0, 2), shapes=DEFAULT_SHAPES) -> TunedSchedule:
    """Cheapest (fixed_cycles, extrapolate) for workload ``w`` whose relative
    L2 velocity error after ``steps`` steps is below target / margin; then
    the faster tiling mode and the fastest launch shape for it."""
    key = size_class(w)
    if use_cache and key in _CACHE:
        return _CACHE[key]

    def ref_setup(sp):
        sp.fixed_cycles = 0
        sp.tol = ref_tol
        sp.max_cycles = 200

    vref, _ = _run(w, steps, ref_setup)
    nref = float(torch.linalg.vector_norm(vref))
    trials = []
    best = None
    for cycles, order in candidates:
        def setup(sp, cycles=cycles, order=order):
            sp.fixed_cycles = cycles
            sp.extrapolate = order
        vel, ms = _run(w, steps, setup)
        err = float(torch.linalg.vector_norm(vel - vref)) / (nref if nref > 0 else 1.0)
        trials.append({"fixed_cycles": cycles, "extrapolate": order, "ms_per_step": ms,
                       "vel_err": err})
        if err * margin <= target and (best is None or ms < best[2]):
            best = (cycles, order, ms, err)
    if best is None:   # nothing met the target: the most accurate candidate
        t = min(trials, key=lambda r: r["vel_err"])
        best = (t["fixed_cycles"], t["extrapolate"], t["ms_per_step"], t["vel_err"])
    # tiling mode on the winning schedule: best of two timed runs each
    tiling_ms = {}
    for variant in tilings:
        def tsetup(sp, variant=variant):
            sp.fixed_cycles = best[0]
            sp.extrapolate = best[1]
            sp.variant = variant
        tiling_ms[variant] = min(_run(w, steps, tsetup)[1] for _ in range(2))
    var = min(tiling_ms, key=tiling_ms.get) if tiling_ms else 0
    ms = tiling_ms.get(var, best[2])
    # launch shape on the winning schedule and tiling mode (the cooperative
    # lower cycle exists for variant 0 only)
    shape_ms = {}
    for shape in shapes:
        if shape[2] and var != 0:
            continue
        def ssetup(sp, shape=shape):
            sp.fixed_cycles = best[0]
            sp.extrapolate = best[1]
            sp.variant = var
            sp.component_streams, sp.launch_overlap, sp.lower_cycle = shape
        shape_ms[shape] = min(_run(w, steps, ssetup)[1] for _ in range(2))
    shape = min(shape_ms, key=shape_ms.get) if shape_ms else TunedSchedule.shape
    if shape_ms:
        ms = shape_ms[shape]
    out = TunedSchedule(best[0], best[1], ms, best[3], trials, var, tiling_ms, shape, shape_ms)
    if use_cache:
        _CACHE[key] = out
    return out


def apply(sim, schedule: TunedSchedule):
    """Set a tuned schedule on a simulation's solver."""
    sp = sim.solver_params()
    sp.fixed_cycles = schedule.fixed_cycles
    sp.extrapolate = schedule.extrapolate
    sp.variant = schedule.variant
    sp.component_streams, sp.launch_overlap, sp.lower_cycle = schedule.shape
    V.vsv_set_solver(sim.g, sp)
