"""The single-launch lower V-cycle: the levels below the finest in one
cooperative launch with bounded grid barriers.  It must give the iterates of
the level-by-level reference kernels bit for bit, in both precisions and for
every boundary kind, and its barrier waits must end by themselves: a barrier
that expects an arrival which never comes reports a timeout instead of
hanging, and the grid stays usable afterwards."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_05031_gb300 import build
    build.build()
    from paper_2601_05031_gb300 import vsv
    vsv.lib()
    return vsv


def _solve(V, shape, prec, bc, variant, lower, shift=0.0, cycles=3, seed=31):
    from paper_2601_05031_gb300.sim import Simulation
    nz, ny, nx = shape
    b = inputs.random_field(shape, seed=seed)
    sim = Simulation(nx, ny, nz, 1.0, prec)
    sp = sim.solver_params()
    sp.variant = variant
    sp.lower_cycle = lower
    V.vsv_set_solver(sim.g, sp)
    launches0 = sim.kernel_launches()
    x, cyc, rr, st = sim.solve_poisson(b, periodic=bc, tol=0.0, max_cycles=cycles, check=False,
                                       shift=shift)
    n = sim.kernel_launches() - launches0
    assert V.vsv_check(sim.g, check=False) == V.VSV_OK
    sim.close()
    return x, n


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("bc,shift", [((True, False, True), 0.0), ((True, False, False), 0.0),
                                      ((True, False, False), 2.5)])
def test_single_launch_lower_cycle_bit_identical(V, prec, bc, shift):
    """128 x 64 x 48 (levels 64 x 32 x 24, 32 x 16 x 12, ...): the lower
    levels do not fit one CTA, so the forced single launch runs levels 1 and
    2 grid-wide and the rest as the one-CTA coarse cycle.  Same bits as the
    reference per-colour kernels (variant 1), with fewer launches than the
    level-by-level fast path."""
    shape = (48, 64, 128)
    p = V.VSV_MIXED if prec == "mixed" else V.VSV_FP64
    x_ref, _ = _solve(V, shape, p, bc, 1, 0, shift)
    x_one, n_one = _solve(V, shape, p, bc, 0, 1, shift)
    x_lvl, n_lvl = _solve(V, shape, p, bc, 0, 0, shift)
    assert np.array_equal(x_one, x_ref)
    assert np.array_equal(x_lvl, x_ref)
    assert n_one < n_lvl, (n_one, n_lvl)
    assert np.all(np.isfinite(x_one)) and np.max(np.abs(x_one)) > 0


def test_single_launch_lower_cycle_in_time_steps(V):
    """A mixed vesicle in Couette flow, 128 x 64 x 64, fixed-cycle steps:
    the forced single launch and the level-by-level lower levels give the
    same phi and velocity bits after a few steps (also through the captured
    graph of a one-grid batch)."""
    import torch
    from paper_2601_05031_gb300.sim import Simulation, Batch
    w = inputs.vesicle(128, 64, 64, inputs.COUETTE, 0.9, 1.5, dt=1e-4, b_range=(0.2, 0.24))
    out = []
    for lower in (1, 0):
        sim = Simulation.from_workload(w, V.VSV_MIXED, stream=torch.cuda.Stream())
        sp = sim.solver_params()
        sp.fixed_cycles = 3
        sp.lower_cycle = lower
        V.vsv_set_solver(sim.g, sp)
        sim.set_phi(w.phi0)
        sim.step(3, w.dt)
        b = Batch([sim])
        b.step(6, w.dt)
        b.close()
        assert V.vsv_check(sim.g, check=False) == V.VSV_OK
        out.append([sim.field(V.VSV_FIELD_PHI)] +
                   [sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)])
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_grid_barrier_completes_and_its_bound_runs_out(V):
    """The bounded grid barrier: with every CTA arriving, 20 barriers
    complete; expecting one arrival more than the launch has (an arrival that
    never comes), every wait gives up after 20 ms, the call reports the
    timeout, and the grid's next solve is unaffected."""
    import time
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation(64, 32, 32, 1.0, V.VSV_MIXED)
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert V.vsv_barrier_check(sim.g, sms, 20, 0, 1000.0) == V.VSV_OK
    t0 = time.perf_counter()
    st = V.vsv_barrier_check(sim.g, sms, 3, 1, 20.0)
    dt = time.perf_counter() - t0
    assert st == V.VSV_ECUDA, st
    assert "ran out of time" in V.vsv_last_error(sim.g)
    assert dt < 5.0, dt
    # the status bit was cleared: the grid works on
    assert V.vsv_check(sim.g, check=False) == V.VSV_OK
    assert V.vsv_barrier_check(sim.g, 2, 5, 0, 1000.0) == V.VSV_OK
    b = inputs.random_field((32, 32, 64), seed=5)
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, True), tol=1e-8, max_cycles=30,
                                       check=False)
    assert st == V.VSV_OK and rr <= 1e-8
    # arguments are checked before any launch
    assert V.vsv_barrier_check(sim.g, 0, 1, 0, 10.0) == V.VSV_EINVAL
    assert V.vsv_barrier_check(sim.g, 10 ** 6, 1, 0, 10.0) == V.VSV_EINVAL
    assert V.vsv_barrier_check(sim.g, 2, 1, 0, 0.0) == V.VSV_EINVAL
    sim.close()


def test_fused_sweep_copy_wait_bound_runs_out(V):
    """The fused sweep's waits for its bulk-copied planes are bounded: with
    every copy group expecting bytes that no copy delivers, each wait gives
    up after 20 ms, the call reports the timeout, and the grid's next solve
    (through the same fused sweep) is unaffected."""
    import time
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation(128, 32, 32, 1.0, V.VSV_MIXED)
    t0 = time.perf_counter()
    st = V.vsv_copy_wait_check(sim.g, 4096, 20.0)
    dt = time.perf_counter() - t0
    assert st == V.VSV_ECUDA, st
    assert "ran out of time" in V.vsv_last_error(sim.g)
    assert dt < 5.0, dt
    assert V.vsv_check(sim.g, check=False) == V.VSV_OK
    b = inputs.random_field((32, 32, 128), seed=7)
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, True), tol=1e-6, max_cycles=30,
                                       check=False)
    assert st == V.VSV_OK and rr <= 1e-6
    # arguments and grids the sweep does not serve are refused before any launch
    assert V.vsv_copy_wait_check(sim.g, 10, 20.0) == V.VSV_EINVAL
    assert V.vsv_copy_wait_check(sim.g, 4096, 0.0) == V.VSV_EINVAL
    sim.close()
    sim = Simulation(64, 32, 32, 1.0, V.VSV_MIXED)
    assert V.vsv_copy_wait_check(sim.g, 4096, 20.0) == V.VSV_EINVAL
    sim.close()
    sim = Simulation(128, 32, 32, 1.0, V.VSV_FP64)
    assert V.vsv_copy_wait_check(sim.g, 4096, 20.0) == V.VSV_EINVAL
    sim.close()
