"""GPU parity of the inertial variant (SM eq. 36): the shifted operator
L_h - s of the backward-Euler vorticity step, standalone and inside time
steps, against the CPU oracle on the same seeded inputs."""
import math

import numpy as np
import pytest

import inputs
import oracle
from oracle.poisson import solve_poisson

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


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _sim(V, w, prec, tol, **kw):
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, prec)
    sp = sim.solver_params()
    sp.tol = tol
    for k, v in kw.items():
        setattr(sp, k, v)
    V.vsv_set_solver(sim.g, sp)
    return sim


@pytest.mark.parametrize("shape,bc", [((16, 8, 12), (True, False, False)),
                                      ((16, 10, 8), (True, False, True)),
                                      ((8, 8, 8), (True, True, True))])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shifted_solve_vs_oracle(V, shape, bc, prec):
    """(L_h - s) x = b through vsv_solve_poisson, including the all-periodic
    case that only the shift makes non-singular."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = shape
    P = V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED
    sim = Simulation(nx, ny, nz, 0.8, P)
    b = inputs.random_field((nz, ny, nx), seed=12)
    s = 2.5
    ref = solve_poisson(b, 0.8, bc, s)
    tol = 1e-13 if prec == "fp64" else 1e-11
    x, cyc, rr, st = sim.solve_poisson(b, periodic=bc, tol=tol, max_cycles=200, shift=s)
    assert st == V.VSV_OK and rel(x, ref) < (1e-10 if prec == "fp64" else 1e-9), (rel(x, ref), cyc)
    sim.close()


def test_shifted_solve_bit_identical_across_variants(V):
    """The shift enters every kernel (fused sweeps, tiled defect and
    transfers, one-CTA coarse cycle) with the arithmetic of the reference
    kernels: the two solver variants agree bit for bit."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = 256, 32, 24
    b = inputs.random_field((nz, ny, nx), seed=23)
    out = []
    for variant in (0, 1):
        sim = Simulation(nx, ny, nz, 1.0, V.VSV_MIXED)
        sp = sim.solver_params()
        sp.variant = variant
        V.vsv_set_solver(sim.g, sp)
        x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, True), tol=0.0,
                                           max_cycles=3, check=False, shift=0.7)
        out.append(x)
        sim.close()
    assert np.array_equal(out[0], out[1])
    ref = solve_poisson(b, 1.0, (True, False, True), 0.7)
    assert rel(out[0], ref) < 1e-2


def test_negative_shift_rejected(V):
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation(8, 8, 8, 1.0, V.VSV_FP64)
    b = np.zeros((8, 8, 8))
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, False), check=False, shift=-1.0)
    assert st == V.VSV_EINVAL
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, True, True), check=False, shift=0.0)
    assert st == V.VSV_EINVAL
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inertial_vorticity_decay_closed_form(V, prec):
    """No body, walls at rest: a vorticity eigenmode set as the perturbation
    decays by s / (s - lambda) per step, psi = -omega / lambda."""
    nx, ny, nz = 32, 16, 16
    w = inputs.droplet_duct(nx=nx, ny=ny, nz=nz, radius=3.0, u_max=0.0,
                            flow_kind=inputs.QUIESCENT)
    w.phi0 = np.ones((nz, ny, nx))
    w.eta, w.rho, dt = 0.7, 0.05, 0.01   # dt inside the explicit phi bound; s ~ 7
    P = V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED
    sim = _sim(V, w, P, 1e-13 if prec == "fp64" else 1e-11)
    sim.set_phi(w.phi0)
    tx, ty, tz = 2 * math.pi / nx, 2 * math.pi / (ny + 1), math.pi / (nz + 1)
    u = (np.sin(tz * (np.arange(nz) + 1))[:, None, None]
         * np.sin(ty * (np.arange(ny) + 1))[None, :, None]
         * np.cos(tx * np.arange(nx) + 0.3)[None, None, :])
    lam = sum(2 * math.cos(t) - 2 for t in (tx, ty, tz))
    amp = (0.3, -0.1, 0.2)
    for c in range(3):
        sim.set_field(V.VSV_FIELD_OMEGA_PERT_X + c, amp[c] * u)
    s = w.rho / (w.eta * dt)
    g = s / (s - lam)
    sim.step(2, dt)
    lim = 1e-10 if prec == "fp64" else 1e-9
    for c in range(3):
        om = sim.field(V.VSV_FIELD_OMEGA_PERT_X + c)
        ps = sim.field(V.VSV_FIELD_PSI_PERT_X + c)
        want = amp[c] * g ** 2 * u
        assert rel(om, want) < lim, (c, rel(om, want))
        assert rel(ps, -want / lam) < lim, (c, rel(ps, -want / lam))
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inertial_steps_vs_oracle(V, prec):
    """A droplet in duct flow with rho > 0: phi, omega, psi and the velocity
    after three backward-Euler vorticity steps against the oracle."""
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5, dt=0.01)
    w.rho = 1.0
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(3):
        oracle.step(st, w.dt)
    P = V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED
    sim = _sim(V, w, P, 1e-13 if prec == "fp64" else 1e-11)
    sim.set_phi(w.phi0)
    sim.step(3, w.dt)
    # FP64: the 1e-10 bar; mixed: phi and the full fields far below 1e-6, the
    # velocity (differences of psi') at the 1e-6 bar of the mixed path
    lim = 1e-10 if prec == "fp64" else 1e-9
    lim_v = 1e-10 if prec == "fp64" else 1e-6
    assert rel(sim.field(V.VSV_FIELD_PHI), st.phi) < lim
    om = np.stack([sim.field(V.VSV_FIELD_OMEGA_X + c) for c in range(3)])
    ps = np.stack([sim.field(V.VSV_FIELD_PSI_X + c) for c in range(3)])
    vel = np.stack([sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)])
    assert rel(om, np.stack(st.omega)) < 10 * lim
    assert rel(ps, np.stack(st.psi)) < lim
    assert rel(vel, np.stack(oracle.velocity(st))) < lim_v
    # the inertial term matters: the non-inertial oracle differs by far more
    st0 = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    st0.p.rho = 0.0
    for _ in range(3):
        oracle.step(st0, w.dt)
    assert rel(np.stack(st0.omega), np.stack(st.omega)) > 1e3 * lim
    sim.close()
