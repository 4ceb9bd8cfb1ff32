"""Plain, slow FP64 CPU oracle of the vorticity--stream-vector phase-field step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it, and this package never imports the product path.

What it computes (Gallen et al., "Deformable bodies in a 3-dimensional
viscous flow: vorticity-stream vector formulation"):

* the coupled system of main-text eqs. gen2, gen1, gen3 (= SM eq. 29):
  d(phi)/dt = M (lap mu + lambda_V) - (curl psi) . grad phi,
  lap omega = (1/eta) grad phi x grad mu,   lap psi = -omega;
* forward Euler for phi and the segregated order of the numerical-
  implementation section: advance phi, then solve omega, then psi;
* mu from the Cahn-Hilliard energy (eq. 31 / SM 1c) or the phase-field
  Helfrich energy (eq. 30, derivative SM eq. 35), area functional SM eq. 32,
  volume penalty SM eqs. 37-38;
* Dirichlet wall data for omega and psi taken from the body-free flow
  (boundary-conditions section), periodic flow axis;
* the in-plane stress of the in-plane-shear section and the flow observables
  of the results section.

Poisson problems are solved exactly (sparse direct solve of the assembled
7-point matrix, or its exact eigen-decomposition by sine / Fourier
transforms), so the oracle's answer does not depend on a solver tolerance.

Parity status per function is stated in each module header; the functions
whose results are pinned by ``tests/test_oracle_pins.py`` are listed there.
"""
from .grid import (GridSpec, pad_flow, pad_mirror, lap, grad, curl, lap_mirror,
                   grad_mirror)
from .poisson import poisson_matrix, solve_poisson, solve_poisson_dense, apply_poisson
from .flow import BaseFlow, base_flow
from .free_energy import (chem_potential, volume, area, area_density, helfrich_energy,
                          ch_energy, prefactor_cf)
from .step import OracleParams, OracleState, init_state, step, velocity, params_from_workload
from .diagnostics import diagnostics

__all__ = [
    "GridSpec", "pad_flow", "pad_mirror", "lap", "grad", "curl", "lap_mirror", "grad_mirror",
    "poisson_matrix", "solve_poisson", "solve_poisson_dense", "apply_poisson",
    "BaseFlow", "base_flow", "chem_potential", "volume", "area", "area_density",
    "helfrich_energy", "ch_energy", "prefactor_cf", "OracleParams", "OracleState",
    "init_state", "step", "velocity", "params_from_workload", "diagnostics",
]
