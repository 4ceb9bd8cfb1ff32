"""Time-dependent walls on the GPU (supplementary material, the
time-dependency paragraph after eq. 36): the GPU path through the C ABI
against the oracle, which pins these flows to their closed forms, on the same
seeded inputs.  FP64 path: relative L2 <= 1e-10 on phi and velocity, mixed
path: <= 1e-6 (with converged solves 1e-8)."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu

MOTION = ((0.3, -0.2), (0.02, 0.035), (40.0, 25.0), (0.4, -1.1))   # ramp, amp, freq, phase


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


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _sim(V, w, prec, tol=None, fixed=0, stream=None):
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, prec, stream=stream)
    sp = sim.solver_params()
    if tol is not None:
        sp.tol = tol
    sp.fixed_cycles = fixed
    V.vsv_set_solver(sim.g, sp)
    return sim


def _vel(V, sim):
    return [sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)]


def _vrel(a, b):
    num = sum(np.sum((a[c] - b[c]) ** 2) for c in range(3))
    den = sum(np.sum(b[c] ** 2) for c in range(3))
    return float(np.sqrt(num / den))


def test_body_free_oscillating_couette_every_step(V):
    """No body: the GPU velocity is the linear profile of each step's wall
    speeds (the oracle's, pinned to the closed form), FP64 and mixed."""
    w = inputs.droplet_duct(nx=16, ny=12, nz=8, radius=3.0, dt=0.01, flow_kind=inputs.COUETTE)
    w.u_max, w.v_lo, w.v_hi = 0.0, -0.05, 0.05
    w.phi0 = np.ones_like(w.phi0)
    w.wall_motion = MOTION
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    sims = [_sim(V, w, V.VSV_FP64, tol=1e-13), _sim(V, w, V.VSV_MIXED, tol=1e-10)]
    for s in sims:
        s.set_phi(w.phi0)
    for n in range(5):
        ov = oracle.velocity(st)
        for s, tol in zip(sims, (1e-13, 1e-9)):
            assert _vrel(_vel(V, s), ov) < tol, (n, _vrel(_vel(V, s), ov))
            d = s.diagnostics()
            assert abs(d["time"] - st.t) < 1e-15
        oracle.step(st, w.dt)
        for s in sims:
            s.step(1, w.dt)
    for s in sims:
        s.close()


@pytest.mark.parametrize("kind", ["couette", "duct"])
def test_vesicle_with_moving_walls_against_oracle(V, kind):
    """A Helfrich vesicle in oscillating Couette flow (both walls moving)
    or in a duct whose Poiseuille speed ramps and oscillates: four steps,
    FP64 within 1e-10 of the oracle and mixed (converged solves) within 1e-8,
    phi and velocity at every step.  Measured on GB300 (Couette): FP64
    velocity 5e-14, mixed 9e-10 .. 2.9e-9, the same level as with steady
    walls (8e-10 .. 1.7e-9): the mixed path's floor here, from the FP32
    rounding that the Helfrich operator amplifies in mu and the source."""
    if kind == "couette":
        w = inputs.vesicle(32, 16, 16, inputs.COUETTE, 0.9, 1.0, dt=5e-4, b_range=(0.24, 0.28))
        w.wall_motion = MOTION
    else:
        w = inputs.vesicle(32, 16, 16, inputs.POISEUILLE_DUCT, 0.9, 1.0, dt=5e-4,
                           b_range=(0.24, 0.28))
        w.wall_motion = ((0.5, 0.0), (0.02, 0.0), (30.0, 0.0), (0.2, 0.0))
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    s64 = _sim(V, w, V.VSV_FP64, tol=1e-13)
    smx = _sim(V, w, V.VSV_MIXED, tol=1e-12)
    for s in (s64, smx):
        s.set_phi(w.phi0)
    for n in range(4):
        oracle.step(st, w.dt)
        s64.step(1, w.dt)
        smx.step(1, w.dt)
        ov = oracle.velocity(st)
        assert rel(s64.field(V.VSV_FIELD_PHI), st.phi) < 1e-10
        assert _vrel(_vel(V, s64), ov) < 1e-10, (n, _vrel(_vel(V, s64), ov))
        assert rel(smx.field(V.VSV_FIELD_PHI), st.phi) < 1e-9
        assert _vrel(_vel(V, smx), ov) < 1e-8, (n, _vrel(_vel(V, smx), ov))
    s64.close()
    smx.close()


def test_moving_walls_graph_replay_state_and_steady_reset(V):
    """The captured step graph carries the wall time on the device: six
    replayed steps give the bits of six plain steps.  A state saved and
    restored continues bit for bit (the walls of the restored time), and
    steady walls again reproduce a grid that never moved."""
    import ctypes
    import torch
    from paper_2601_05031_gb300.sim import Batch
    w = inputs.vesicle(64, 32, 32, inputs.COUETTE, 0.9, 1.0, dt=5e-4, b_range=(0.24, 0.28))
    w.wall_motion = MOTION
    out = []
    for use_graph in (False, True):
        s = _sim(V, w, V.VSV_MIXED, fixed=3, stream=torch.cuda.Stream())
        s.set_phi(w.phi0)
        s.step(3, w.dt)
        if use_graph:
            b = Batch([s])
            b.step(6, w.dt)
            b.close()
        else:
            s.step(6, w.dt)
        out.append([s.field(V.VSV_FIELD_PHI)] + _vel(V, s))
        s.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    # state round trip in the middle of the motion
    s = _sim(V, w, V.VSV_MIXED, fixed=3)
    s.set_phi(w.phi0)
    s.step(4, w.dt)
    nb = V.lib().vsv_state_bytes(s.g)
    blob = (ctypes.c_char * nb)()
    V.vsv_get_state(s.g, ctypes.addressof(blob), nb)
    s.step(3, w.dt)
    a = [s.field(V.VSV_FIELD_PHI)] + _vel(V, s)
    V.vsv_set_state(s.g, ctypes.addressof(blob), nb)
    s.step(3, w.dt)
    b = [s.field(V.VSV_FIELD_PHI)] + _vel(V, s)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # back to steady walls: the same bits as a grid that never had motion
    V.vsv_set_wall_motion(s.g, None)
    s.set_phi(w.phi0)
    s.step(3, w.dt)
    c = [s.field(V.VSV_FIELD_PHI)] + _vel(V, s)
    s.close()
    w.wall_motion = None
    t = _sim(V, w, V.VSV_MIXED, fixed=3)
    t.set_phi(w.phi0)
    t.step(3, w.dt)
    d = [t.field(V.VSV_FIELD_PHI)] + _vel(V, t)
    t.close()
    for x, y in zip(c, d):
        assert np.array_equal(x, y)


def test_wall_motion_argument_checks(V):
    from paper_2601_05031_gb300.sim import Simulation
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5, dt=0.01, u_max=0.0,
                            flow_kind=inputs.QUIESCENT)
    s = Simulation.from_workload(w, V.VSV_FP64)
    assert V.vsv_set_wall_motion(s.g, MOTION, check=False) == V.VSV_EINVAL   # quiescent
    assert V.vsv_set_wall_motion(s.g, None, check=False) == V.VSV_OK
    s.close()
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5, dt=0.01)
    s = Simulation.from_workload(w, V.VSV_FP64)
    # wall 1 only moves in Couette flow
    assert V.vsv_set_wall_motion(s.g, MOTION, check=False) == V.VSV_EINVAL
    bad = ((float("nan"), 0.0), (0.0, 0.0), (0.0, 0.0), (0.0, 0.0))
    assert V.vsv_set_wall_motion(s.g, bad, check=False) == V.VSV_EINVAL
    ok = ((0.1, 0.0), (0.01, 0.0), (5.0, 0.0), (0.0, 0.0))
    assert V.vsv_set_wall_motion(s.g, ok, check=False) == V.VSV_OK
    # the adjoint tape needs steady walls
    import ctypes
    tape = V.vsv_tape_create(s.g, 2, 0.0)
    phi0 = np.ascontiguousarray(w.phi0)
    st = V.lib().vsv_tape_forward(tape, ctypes.c_void_p(phi0.ctypes.data), V.VSV_DTYPE_F64, 0, 2,
                                  w.dt)
    assert st == V.VSV_EINVAL
    V.vsv_tape_destroy(tape)
    s.close()
    # and an inertial flow refuses it
    w.rho = 0.5
    s = Simulation.from_workload(w, V.VSV_FP64)
    assert V.vsv_set_wall_motion(s.g, ok, check=False) == V.VSV_EINVAL
    s.close()
