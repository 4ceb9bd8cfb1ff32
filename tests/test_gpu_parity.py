"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  FP64 path: relative L2 <= 1e-10 on phi and velocity;
mixed path: <= 1e-6 (tolerances of the hot-path specification)."""
import ctypes
import math

import numpy as np
import pytest

import inputs
import oracle
from oracle.poisson import solve_poisson_dense, solve_poisson

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


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


def make_sim(V, w, prec, tol=None, kind=None, fixed=0, **kw):
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, prec)
    sp = sim.solver_params()
    if tol is not None:
        sp.tol = tol
    if kind is not None:
        sp.kind = kind
    sp.fixed_cycles = fixed
    for k, v in kw.items():
        setattr(sp, k, v)
    V.vsv_set_solver(sim.g, sp)
    return sim


# ------------------------------------------------------------ workloads
def small_droplet():
    return inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5, dt=0.01)


def small_vesicle(kind, nx=32, ny=16, nz=16, eps=1.0, vr=0.9, dt=5e-4):
    w = inputs.vesicle(nx, ny, nz, kind, vr, eps, dt=dt, b_range=(0.24, 0.28), k_area=0.05)
    return w


WORKLOADS = {
    "droplet_duct": small_droplet,
    "vesicle_couette": lambda: small_vesicle(inputs.COUETTE),
    "vesicle_planar": lambda: small_vesicle(inputs.POISEUILLE_PLANAR),
    "vesicle_duct": lambda: small_vesicle(inputs.POISEUILLE_DUCT),
    "droplet_quiescent": lambda: inputs.droplet_duct(nx=16, ny=10, nz=12, radius=3.0, u_max=0.0,
                                                     flow_kind=inputs.QUIESCENT),
}


def oracle_fields(st):
    v = oracle.velocity(st)
    return {"phi": st.phi, "mu": st.mu, "omega": st.omega, "psi": st.psi, "vel": list(v)}


def gpu_fields(V, sim):
    F = {"phi": sim.field(V.VSV_FIELD_PHI), "mu": sim.field(V.VSV_FIELD_MU)}
    F["omega"] = [sim.field(V.VSV_FIELD_OMEGA_X + c) for c in range(3)]
    F["psi"] = [sim.field(V.VSV_FIELD_PSI_X + c) for c in range(3)]
    F["vel"] = [sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)]
    return F


def field_errors(G, O):
    e = {"phi": rel(G["phi"], O["phi"]), "mu": rel(G["mu"], O["mu"])}
    for key in ("omega", "psi", "vel"):
        e[key] = rel(np.stack(G[key]), np.stack(O[key]))
    return e


# ------------------------------------------------------------ Poisson
BCS = [((16, 8, 12), (True, False, False)), ((16, 10, 8), (True, False, True)),
       ((12, 9, 7), (False, False, False)), ((1, 16, 16), (True, False, False)),
       ((24, 6, 10), (True, True, False))]


@pytest.mark.parametrize("shape,bc", BCS)
@pytest.mark.parametrize("prec,kind", [("fp64", "mg"), ("fp64", "sor"), ("mixed", "mg")])
def test_poisson_vs_oracle(V, shape, bc, prec, kind):
    nx, ny, nz = shape
    if nx > 1 and nx % 2 and bc[0]:
        pytest.skip("odd periodic")
    from paper_2601_05031_gb300.sim import Simulation
    P = V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED
    sim = Simulation(nx, ny, nz, 0.8, P)
    sp = sim.solver_params()
    sp.kind = V.VSV_SOLVER_SOR if kind == "sor" else V.VSV_SOLVER_MG
    V.vsv_set_solver(sim.g, sp)
    b = inputs.random_field((nz, ny, nx), seed=11)
    ref = solve_poisson_dense(b, 0.8, bc)
    tol = 1e-13 if prec == "fp64" else 1e-11
    x, cyc, rr, st = sim.solve_poisson(b, periodic=bc, tol=tol, max_cycles=20000)
    lim = FP64_TOL if prec == "fp64" else MIXED_TOL
    assert rel(x, ref) < lim, (rel(x, ref), cyc, rr)
    sim.close()


def test_poisson_manufactured_eigenvector(V):
    """C-P1 on the GPU: sin-product eigenvector recovered by the FP64 MG."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz, h = 32, 24, 16, 1.0
    sim = Simulation(nx, ny, nz, h, V.VSV_FP64)
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    tx, ty, tz = 2 * math.pi * 3 / nx, math.pi * 2 / (ny + 1), math.pi * 1 / (nz + 1)
    u = (np.sin(tz * (k + 1))[:, None, None] * np.sin(ty * (j + 1))[None, :, None]
         * np.cos(tx * i + 0.2)[None, None, :])
    lam = sum(2 * math.cos(t) - 2 for t in (tx, ty, tz)) / h ** 2
    x, cyc, rr, st = sim.solve_poisson(lam * u, periodic=(True, False, False), tol=1e-13)
    assert rel(x, u) < 1e-11, (rel(x, u), cyc, rr)
    sim.close()


def test_mixed_defect_correction_reaches_fp64_class_accuracy(V):
    """Outer defect correction with the double-word iterate: FP32 V-cycles
    on the correction, the exact defect and x += e in double-word arithmetic
    take the relative residual and the error far below FP32 rounding."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = 64, 32, 32
    sim = Simulation(nx, ny, nz, 1.0, V.VSV_MIXED)
    b = inputs.random_field((nz, ny, nx), seed=5)
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, False), tol=1e-12,
                                       max_cycles=60, check=False)
    ref = solve_poisson(b, 1.0, (True, False, False))
    assert st == V.VSV_OK and rr <= 1e-12, (st, rr, cyc)
    assert rel(x, ref) < 1e-10, rel(x, ref)
    sim.close()


# ------------------------------------------------------------ initial state
@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_initial_state_fp64(V, name):
    w = WORKLOADS[name]()
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    sim = make_sim(V, w, V.VSV_FP64, tol=1e-13)
    sim.set_phi(w.phi0)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    for key, val in e.items():
        assert val < FP64_TOL, (key, e)
    sim.close()


# ------------------------------------------------------------ time steps
@pytest.mark.parametrize("name,nsteps", [("droplet_duct", 5), ("vesicle_couette", 4),
                                         ("vesicle_planar", 3), ("vesicle_duct", 3),
                                         ("droplet_quiescent", 4)])
def test_steps_fp64(V, name, nsteps):
    w = WORKLOADS[name]()
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(nsteps):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_FP64, tol=1e-13)
    sim.set_phi(w.phi0)
    sim.step(nsteps, w.dt)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    assert e["phi"] < FP64_TOL and e["vel"] < FP64_TOL, e
    for key in ("mu", "omega", "psi"):
        assert e[key] < 1e-9, (key, e)
    sim.close()


def test_droplet_24x24x48_sor_fp64(V):
    """The plain-FP64 droplet workload: 48x24x24 duct, red-black SOR to a
    relative residual of 1e-13 (tighter than the 1e-10 it asks for, so that
    the discrete answer, not the stopping point, is compared), 10 steps."""
    w = inputs.droplet_24x24x48()
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(w.nsteps):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_FP64, tol=1e-13, kind=V.VSV_SOLVER_SOR, max_cycles=20000,
                   check_every=10)
    sim.set_phi(w.phi0)
    sim.step(w.nsteps, w.dt)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    assert e["phi"] < FP64_TOL and e["vel"] < FP64_TOL, e
    sim.close()


@pytest.mark.parametrize("name,nsteps", [("droplet_duct", 5), ("vesicle_couette", 4),
                                         ("vesicle_duct", 3)])
def test_steps_mixed(V, name, nsteps):
    w = WORKLOADS[name]()
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(nsteps):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_MIXED, tol=1e-10)
    sim.set_phi(w.phi0)
    sim.step(nsteps, w.dt)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    assert e["phi"] < MIXED_TOL and e["vel"] < MIXED_TOL, e
    sim.close()


def test_fixed_cycle_schedule_matches_converged(V):
    """Mixed path with a fixed two-V-cycle schedule per solve (the launch
    configuration of the benchmark) stays within 1e-6 of the oracle."""
    w = small_vesicle(inputs.COUETTE, nx=64, ny=32, nz=32, eps=1.5, dt=1e-4)
    nsteps = 20
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(nsteps):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_MIXED, tol=1e-8, fixed=2)
    sim.set_phi(w.phi0)
    sim.step(nsteps, w.dt)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    assert e["phi"] < MIXED_TOL and e["vel"] < MIXED_TOL, e
    sim.close()


# ------------------------------------------------------------ degenerate cases
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_no_body_keeps_the_base_flow(V, prec):
    """phi = 1 everywhere (no interface): no source, so omega' and psi' stay
    at the round-off of the tabulated body-free fields, the velocity is the
    body-free Couette profile, and phi does not move."""
    w = small_vesicle(inputs.COUETTE)
    w.phi0 = np.ones_like(w.phi0)
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(2):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED,
                   tol=1e-13 if prec == "fp64" else 1e-11)
    sim.set_phi(w.phi0)
    sim.step(2, w.dt)
    assert np.array_equal(sim.field(V.VSV_FIELD_PHI), w.phi0)
    for c in range(3):
        assert np.max(np.abs(sim.field(V.VSV_FIELD_PSI_PERT_X + c))) < 1e-10
        assert np.max(np.abs(sim.field(V.VSV_FIELD_OMEGA_PERT_X + c))) < 1e-10
    vel = np.stack([sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)])
    assert rel(vel, np.stack(oracle.velocity(st))) < (1e-12 if prec == "fp64" else 1e-7)
    sim.close()


def test_tension_without_bending_vs_oracle(V):
    """Helfrich kind with kappa = 0 and a membrane tension: mu is the
    tension term and the area multiplier alone."""
    w = small_vesicle(inputs.POISEUILLE_DUCT)
    w.kappa, w.sigma = 0.0, 0.5
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(3):
        oracle.step(st, w.dt)
    sim = make_sim(V, w, V.VSV_FP64, tol=1e-13)
    sim.set_phi(w.phi0)
    sim.step(3, w.dt)
    e = field_errors(gpu_fields(V, sim), oracle_fields(st))
    assert max(e.values()) < 1e-10, e
    sim.close()


def test_zero_steps_is_a_no_op(V):
    w = small_droplet()
    sim = make_sim(V, w, V.VSV_MIXED, fixed=2)
    sim.set_phi(w.phi0)
    sim.step(1, w.dt)
    before = [sim.field(f) for f in (V.VSV_FIELD_PHI, V.VSV_FIELD_PSI_PERT_X, V.VSV_FIELD_MU)]
    d0 = sim.diagnostics()
    assert V.vsv_step(sim.g, 0, w.dt) == V.VSV_OK
    after = [sim.field(f) for f in (V.VSV_FIELD_PHI, V.VSV_FIELD_PSI_PERT_X, V.VSV_FIELD_MU)]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert sim.diagnostics()["steps"] == d0["steps"]
    sim.close()


# ------------------------------------------------------------ diagnostics
@pytest.mark.parametrize("sigma", [0.0, 0.4])
def test_diagnostics_vs_oracle(V, sigma):
    """All diagnostics against the oracle; with sigma > 0 a membrane tension
    enters the step and the energy (sigma times the face-difference area)."""
    w = small_vesicle(inputs.COUETTE)
    w.sigma = sigma
    st = oracle.init_state(oracle.params_from_workload(w), w.phi0)
    for _ in range(2):
        oracle.step(st, w.dt)
    od = oracle.diagnostics(st)
    sim = make_sim(V, w, V.VSV_FP64, tol=1e-13)
    sim.set_phi(w.phi0)
    sim.step(2, w.dt)
    gd = sim.diagnostics()
    for key in ("volume", "area", "reduced_volume", "energy", "dissipation", "dissipation0",
                "resistance_rel", "omega_dev2", "psi_dev2", "max_sigma_t"):
        assert abs(gd[key] - od[key]) <= 1e-9 * max(1.0, abs(od[key])), (key, gd[key], od[key])
    for a in range(3):
        assert abs(gd["com"][a] - od["com"][a]) < 1e-9
    assert gd["max_div_v"] < 1e-12 and od["max_div_v"] < 1e-12
    assert abs(gd["max_div_psi"] - od["max_div_psi"]) < 1e-9
    prof = sim.stress_profile()
    assert np.max(np.abs(prof - od["stress_profile"])) < 1e-11 * max(1.0, np.abs(od["stress_profile"]).max())
    sig = sim.field(V.VSV_FIELD_STRESS_T)
    assert rel(sig, od["sigma_t"]) < 1e-9
    sim.close()


# ------------------------------------------------------------ state, errors, determinism
def test_state_roundtrip_and_determinism(V):
    w = small_droplet()
    sim = make_sim(V, w, V.VSV_MIXED, fixed=2)
    sim.set_phi(w.phi0)
    sim.step(2, w.dt)
    nb = V.vsv_state_bytes(sim.g)
    blob = np.empty(nb, dtype=np.uint8)
    V.vsv_get_state(sim.g, blob.ctypes.data, nb)
    sim.step(3, w.dt)
    a = sim.field(V.VSV_FIELD_PHI, np.float32)
    V.vsv_set_state(sim.g, blob.ctypes.data, nb)
    sim.step(3, w.dt)
    b = sim.field(V.VSV_FIELD_PHI, np.float32)
    assert np.array_equal(a, b)
    sim2 = make_sim(V, w, V.VSV_MIXED, fixed=2)
    sim2.set_phi(w.phi0)
    sim2.step(5, w.dt)
    assert np.array_equal(a, sim2.field(V.VSV_FIELD_PHI, np.float32))
    sim.close()
    sim2.close()


@pytest.mark.parametrize("field", ["phi", "psi_x"])
def test_fp64_host_transfers_mapped_and_copied(V, field):
    """FP64 words in and out through page-locked host memory (split and
    merged in place by the kernels), through page-locked memory at an
    8-byte offset (the one-word kernels) and through pageable memory (copy
    and staging buffer) give the same bits as the device path."""
    import torch
    w = small_droplet()
    sim = make_sim(V, w, V.VSV_MIXED, fixed=2)
    sim.set_phi(w.phi0)
    sim.step(2, w.dt)
    fid = V.VSV_FIELD_PHI if field == "phi" else V.VSV_FIELD_PSI_PERT_X
    n = w.nx * w.ny * w.nz
    dev = sim.field(fid, np.float64, on_device=True).clone()
    ref = dev.cpu().numpy().ravel()
    # the device path itself: out and back in leaves the state unchanged
    V.vsv_set_field(sim.g, fid, dev.data_ptr(), V.VSV_DTYPE_F64, 1)
    np.testing.assert_array_equal(sim.field(fid, np.float64, on_device=True).cpu().numpy().ravel(), ref)
    pinned = torch.empty(n + 1, dtype=torch.float64, pin_memory=True)
    pageable = np.empty(n + 1, dtype=np.float64)
    for name, buf, off in (("pinned", pinned.data_ptr(), 0), ("pinned+8", pinned.data_ptr(), 8),
                           ("pageable", pageable.ctypes.data, 0),
                           ("pageable+8", pageable.ctypes.data, 8)):
        view = (pinned.numpy() if name.startswith("pinned") else pageable)
        view[:] = np.nan
        assert V.vsv_get_field(sim.g, fid, buf + off, V.VSV_DTYPE_F64, 0) == V.VSV_OK
        got = view[off // 8: off // 8 + n]
        np.testing.assert_array_equal(got, ref, err_msg=name)
        # back in from the same buffer, then out through the device path
        assert V.vsv_set_field(sim.g, fid, buf + off, V.VSV_DTYPE_F64, 0) == V.VSV_OK
        again = sim.field(fid, np.float64, on_device=True).cpu().numpy().ravel()
        np.testing.assert_array_equal(again, ref, err_msg=name)
    sim.close()


def test_error_statuses(V):
    from paper_2601_05031_gb300.sim import Simulation
    w = small_droplet()
    sim = Simulation(w.nx, w.ny, w.nz, 1.0, V.VSV_MIXED)
    assert V.vsv_step(sim.g, 1, 0.01, check=False) == V.VSV_ESTATE
    sim.configure(w)
    sim.set_phi(w.phi0)
    lim = sim.stability_limit()
    assert 0.0119 < lim < 0.0120   # CH bound 2 / (M lam (2 + sigma lam)), lam = 12
    assert V.vsv_step(sim.g, 1, 2 * lim, check=False) == V.VSV_EUNSTABLE
    bad = w.phi0.copy()
    bad[3, 4, 5] = np.nan
    sim.set_field(V.VSV_FIELD_PHI, bad)
    sp = sim.solver_params()
    sp.fixed_cycles = 1
    V.vsv_set_solver(sim.g, sp)
    V.vsv_step(sim.g, 1, w.dt, check=False)
    assert V.vsv_check(sim.g, check=False) == V.VSV_ENONFINITE
    sim.close()


def test_kernel_launch_accounting(V):
    w = small_droplet()
    sim = make_sim(V, w, V.VSV_MIXED, fixed=2)
    sim.set_phi(w.phi0)
    n0 = sim.kernel_launches()
    V.vsv_profile_enable(sim.g, V.VSV_KCLASS_SMOOTH_FINE)
    sim.step(2, w.dt)
    ms, n = V.vsv_profile_read(sim.g, V.VSV_KCLASS_SMOOTH_FINE)
    assert sim.kernel_launches() > n0 and n > 0 and ms > 0
    sim.close()


def test_profile_byte_tally(V):
    """On a tile-aligned grid every finest-level sweep of a correction's
    V(2,2)-cycle is a fused launch: zero-input (8 B/cell), plain (12), plain,
    and the one that updates the double-word iterate (24), for 3 components;
    a step runs the vorticity and the stream-vector solve."""
    nx, ny, nz, cycles = 256, 32, 32, 2
    w = inputs.vesicle_couette_512x256x256(nx=nx, ny=ny, nz=nz, nsteps=1)
    sim = make_sim(V, w, V.VSV_MIXED, fixed=cycles)
    sim.set_phi(w.phi0)
    V.vsv_profile_enable(sim.g, V.VSV_KCLASS_SMOOTH_FINE)
    sim.step(1, w.dt)
    ms, n, nbytes = V.vsv_profile_read(sim.g, V.VSV_KCLASS_SMOOTH_FINE, with_bytes=True)
    sim.close()
    assert n == 2 * cycles * 4
    assert nbytes == 2 * cycles * (8 + 12 + 12 + 24) * nx * ny * nz * 3


def test_step_byte_tally_covers_the_sweeps(V):
    """The always-on tally of a step counts the finest-level sweeps and more
    (defects, transfers, coarse levels, phase kernels)."""
    nx, ny, nz, cycles = 256, 32, 32, 2
    w = inputs.vesicle_couette_512x256x256(nx=nx, ny=ny, nz=nz, nsteps=1)
    sim = make_sim(V, w, V.VSV_MIXED, fixed=cycles)
    sim.set_phi(w.phi0)
    b0 = sim.kernel_bytes()
    sim.step(1, w.dt)
    step_bytes = sim.kernel_bytes() - b0
    sim.close()
    sweeps = 2 * cycles * (8 + 12 + 12 + 24) * nx * ny * nz * 3
    defects = 2 * cycles * 20 * nx * ny * nz * 3
    assert sweeps + defects < step_bytes < 3 * (sweeps + defects)


# ------------------------------------------------------------ fused sweep
@pytest.mark.parametrize("shape,bc", [((256, 32, 24), (True, False, True)),
                                      ((256, 32, 24), (True, False, False)),
                                      ((128, 48, 20), (True, False, False)),
                                      ((256, 32, 24), (True, True, False))])
def test_fused_sweep_bit_identical_to_reference(V, shape, bc):
    """The single-pass fused red-black sweep (variant 0) gives bit-identical
    multigrid iterates to the per-colour reference kernels (variant 1) on a
    tile-aligned grid where it engages (finest and first coarse level): with
    TMA boxes (y walls; z walls or periodic z; one tile across x, whose halo
    groups both wrap onto itself) and, with periodic y, with cp.async
    staging."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = shape
    b = inputs.random_field((nz, ny, nx), seed=21)
    out = []
    for variant in (0, 1):
        sim = Simulation(nx, ny, nz, 1.0, V.VSV_MIXED)
        sp = sim.solver_params()
        sp.variant = variant
        V.vsv_set_solver(sim.g, sp)
        x, cyc, rr, st = sim.solve_poisson(b, periodic=bc, tol=0.0, max_cycles=3, check=False)
        out.append((x, rr))
        sim.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * abs(out[1][1])   # FP32 norm partials, other order
    ref = solve_poisson(b, 1.0, bc)
    assert rel(out[0][0], ref) < 3e-2   # three V-cycles from zero


@pytest.mark.parametrize("shape,bc", [((96, 40, 40), (True, False, False)),
                                      ((200, 24, 32), (True, False, True)),
                                      ((64, 8, 272), (True, True, False))])
def test_ragged_fused_sweep_bit_identical_to_reference(V, shape, bc):
    """Partial edge tiles (extents not multiples of the 128 x 16 tile, and a
    periodic y shorter than the tile): the fused sweep (variant 0) gives the
    iterates of the per-colour reference kernels (variant 1) and of the
    aligned-only fast path (variant 2) bit for bit, and engages (fewer
    launches than variant 2)."""
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = shape
    b = inputs.random_field((nz, ny, nx), seed=31)
    out, launches = [], []
    for variant in (0, 1, 2):
        sim = Simulation(nx, ny, nz, 1.0, V.VSV_MIXED)
        sp = sim.solver_params()
        sp.variant = variant
        V.vsv_set_solver(sim.g, sp)
        l0 = sim.kernel_launches()
        x, cyc, rr, st = sim.solve_poisson(b, periodic=bc, tol=0.0, max_cycles=3, check=False)
        launches.append(sim.kernel_launches() - l0)
        out.append(x)
        sim.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    assert launches[0] < launches[2], launches
    assert np.all(np.isfinite(out[0])) and np.any(out[0] != 0)
    if not bc[1]:
        # three V-cycles from zero (a sanity bound).  With periodic y the
        # short y axis stops the coarsening at a level where the long walled
        # z axis converges slowly; the reference kernels agree bit for bit.
        assert rel(out[0], solve_poisson(b, 1.0, bc)) < 0.1


@pytest.mark.parametrize("kind", ["couette", "duct"])
def test_aligned_fused_steps_bit_identical_to_reference(V, kind):
    """Time steps of a vesicle on a tile-aligned grid (the TMA-staged fused
    sweeps: from zero, with source offsets, with the iterate update fused into
    the last sweep; the Helfrich g formed in the volume / area reduction's
    pass): variants 0 and 1 agree bit for bit."""
    flow = inputs.COUETTE if kind == "couette" else inputs.POISEUILLE_DUCT
    w = inputs.vesicle(256, 32, 32, flow, 0.85, 1.0, dt=1e-4, b_range=(0.25, 0.3))
    assert w.fe_kind == V.VSV_HELFRICH
    res = []
    for variant in (0, 1):
        sim = make_sim(V, w, V.VSV_MIXED, fixed=2, variant=variant)
        sim.set_phi(w.phi0)
        mu0 = sim.field(V.VSV_FIELD_MU)
        sim.step(3, w.dt)
        res.append([mu0, sim.field(V.VSV_FIELD_PHI), sim.field(V.VSV_FIELD_MU)] +
                   [sim.field(V.VSV_FIELD_PSI_PERT_X + c) for c in range(3)])
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_ragged_fused_steps_bit_identical_to_reference(V):
    """Time steps of a vesicle on a grid with partial tiles (source offsets
    in the stream-vector solves, the iterate update fused into the last
    sweep): variants 0 and 1 agree bit for bit."""
    w = inputs.vesicle(96, 40, 40, inputs.POISEUILLE_DUCT, 0.85, 1.0, dt=1e-4,
                       b_range=(0.25, 0.3))
    res = []
    for variant in (0, 1):
        sim = make_sim(V, w, V.VSV_MIXED, fixed=3, variant=variant)
        sim.set_phi(w.phi0)
        sim.step(3, w.dt)
        res.append([sim.field(V.VSV_FIELD_PHI), sim.field(V.VSV_FIELD_MU)] +
                   [sim.field(V.VSV_FIELD_PSI_PERT_X + c) for c in range(3)])
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_droplet_steps_bit_identical_across_variants(V):
    """A Cahn-Hilliard droplet (no Helfrich g, so the volume / area reduction
    stores nothing else): fixed-cycle mixed steps of variants 0 and 1 agree
    bit for bit in phi, mu and psi'."""
    w = small_droplet()
    assert w.fe_kind == V.VSV_CAHN_HILLIARD
    res = []
    for variant in (0, 1):
        sim = make_sim(V, w, V.VSV_MIXED, fixed=2, variant=variant)
        sim.set_phi(w.phi0)
        sim.step(3, w.dt)
        res.append([sim.field(V.VSV_FIELD_PHI), sim.field(V.VSV_FIELD_MU)] +
                   [sim.field(V.VSV_FIELD_PSI_PERT_X + c) for c in range(3)])
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_fused_mixed_solve_vs_oracle(V):
    from paper_2601_05031_gb300.sim import Simulation
    nx, ny, nz = 256, 64, 32
    sim = Simulation(nx, ny, nz, 1.0, V.VSV_MIXED)
    b = inputs.random_field((nz, ny, nx), seed=22)
    x, cyc, rr, st = sim.solve_poisson(b, periodic=(True, False, True), tol=1e-11, max_cycles=40,
                                       check=False)
    ref = solve_poisson(b, 1.0, (True, False, True))
    assert st == V.VSV_OK and rel(x, ref) < 1e-9, (rel(x, ref), cyc, rr)
    sim.close()


@pytest.mark.parametrize("kind", ["couette", "duct", "inertial"])
def test_component_streams_bit_identical(V, kind):
    """Fixed-cycle steps with each component's vorticity and stream-vector
    solves on a stream of its own give the bits of the three components
    together on the grid's stream: over plain steps, and over the replays of
    a captured graph (the component streams fork and join inside it)."""
    import torch
    from paper_2601_05031_gb300.sim import Batch
    flow = inputs.POISEUILLE_DUCT if kind == "duct" else inputs.COUETTE
    w = inputs.vesicle(256, 32, 32, flow, 0.85, 1.0, dt=1e-4, b_range=(0.25, 0.3))
    if kind == "inertial":
        w.rho = 0.5
    res = []
    for cs in (0, 1):
        from paper_2601_05031_gb300.sim import Simulation
        sim = Simulation.from_workload(w, V.VSV_MIXED, stream=torch.cuda.Stream())
        sp = sim.solver_params()
        sp.fixed_cycles = 2
        sp.extrapolate = 2
        sp.component_streams = cs
        V.vsv_set_solver(sim.g, sp)
        sim.set_phi(w.phi0)
        sim.step(4, w.dt)
        b = Batch([sim])
        b.step(6, w.dt)
        b.close()
        assert V.vsv_check(sim.g, check=False) == V.VSV_OK
        res.append([sim.field(V.VSV_FIELD_PHI)] +
                   [sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)] +
                   [sim.field(V.VSV_FIELD_OMEGA_X + c) for c in range(3)])
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("kind,prec,cs", [("couette", "mixed", 0), ("couette", "mixed", 1),
                                          ("duct", "mixed", 1), ("couette", "fp64", 0)])
def test_launch_overlap_bit_identical(V, kind, prec, cs):
    """Steps whose solver and phase-field kernels are launched with
    programmatic stream serialisation (launch_overlap 1: each kernel waits
    for its predecessor inside the kernel) give the bits of plain launches,
    over plain steps and over replays of a captured graph, with and without
    the component streams; and a converged standalone solve (residual-norm
    kernels, host reads between cycles) gives the same iterate.  A value
    outside 0..2 is refused."""
    import torch
    from paper_2601_05031_gb300.sim import Batch, Simulation
    flow = inputs.POISEUILLE_DUCT if kind == "duct" else inputs.COUETTE
    w = inputs.vesicle(256, 32, 32, flow, 0.85, 1.0, dt=1e-4, b_range=(0.25, 0.3))
    p = V.VSV_MIXED if prec == "mixed" else V.VSV_FP64
    rng = np.random.default_rng(11)
    rhs = rng.standard_normal((w.nz, w.ny, w.nx))
    res = []
    for ov in (0, 1):
        sim = Simulation.from_workload(w, p, stream=torch.cuda.Stream())
        sp = sim.solver_params()
        assert sp.launch_overlap == 2   # the default: by grid size
        sp.fixed_cycles = 2
        sp.extrapolate = 2
        sp.component_streams = cs
        sp.launch_overlap = ov
        V.vsv_set_solver(sim.g, sp)
        sim.set_phi(w.phi0)
        sim.step(3, w.dt)
        b = Batch([sim])
        b.step(6, w.dt)
        b.close()
        assert V.vsv_check(sim.g, check=False) == V.VSV_OK
        fields = ([sim.field(V.VSV_FIELD_PHI), sim.field(V.VSV_FIELD_MU)] +
                  [sim.field(V.VSV_FIELD_VEL_X + c) for c in range(3)] +
                  [sim.field(V.VSV_FIELD_PSI_PERT_X + c) for c in range(3)])
        # the standalone solve takes over the grid's workspace (no state after it)
        x, cyc, rr, st = sim.solve_poisson(rhs, periodic=(True, False, True), tol=1e-9)
        assert st == V.VSV_OK and rr <= 1e-9
        res.append(fields + [x, cyc])
        if ov == 1:
            sp.launch_overlap = 3
            with pytest.raises(V.VsvError) as e:
                V.vsv_set_solver(sim.g, sp)
            assert e.value.status == V.VSV_EINVAL
        sim.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_async_host_transfers_of_phi(V):
    """VSV_HOST_ASYNC: FP64 phi set from and read into page-locked host
    memory on the grid's copy streams gives the bits of the synchronous
    calls, in a loop of set / step / get with no synchronisation but one
    vsv_check at the end; for other fields the kind acts synchronously; an
    unknown memory kind is refused."""
    import torch
    from paper_2601_05031_gb300.sim import Simulation
    w = inputs.vesicle(256, 32, 32, inputs.COUETTE, 0.85, 1.0, dt=1e-4, b_range=(0.25, 0.3))
    shape = (w.nz, w.ny, w.nx)
    outs = []
    for kind in (0, V.VSV_HOST_ASYNC):
        sim = make_sim(V, w, V.VSV_MIXED, fixed=2)
        sim.set_phi(w.phi0)
        sim.step(2, w.dt)
        src = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        src.copy_(torch.from_numpy(sim.field(V.VSV_FIELD_PHI)))
        dst = [torch.zeros(shape, dtype=torch.float64, pin_memory=True) for _ in range(3)]
        for n in range(3):
            V.vsv_set_field(sim.g, V.VSV_FIELD_PHI, src.data_ptr(), V.VSV_DTYPE_F64, kind)
            sim.step(1, w.dt)
            V.vsv_get_field(sim.g, V.VSV_FIELD_PHI, dst[n].data_ptr(), V.VSV_DTYPE_F64, kind)
        V.vsv_check(sim.g)
        mu = np.zeros(shape)
        assert V.vsv_get_field(sim.g, V.VSV_FIELD_MU, mu.ctypes.data, V.VSV_DTYPE_F64,
                               V.VSV_HOST_ASYNC) == V.VSV_OK
        assert np.array_equal(mu, sim.field(V.VSV_FIELD_MU))   # acted synchronously
        assert V.lib().vsv_get_field(sim.g, V.VSV_FIELD_PHI, ctypes.c_void_p(dst[0].data_ptr()),
                                     V.VSV_DTYPE_F64, 3) == V.VSV_EINVAL
        outs.append([d.numpy().copy() for d in dst])
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
        assert np.any(a != 0)
