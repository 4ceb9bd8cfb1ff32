"""GPU parity of the discrete adjoint with checkpointing (vsv_tape_*):
gradients of J = h^3/2 sum (phi^N - target)^2 with respect to phi^0, kappa
and sigma against the oracle's adjoint (oracle/adjoint.py) on the same
seeded inputs, against central differences of the GPU forward map, and the
checkpointing invariances (gradient independent of the checkpoint interval,
grid left at phi^N), also for the inertial variant."""
import dataclasses

import numpy as np
import pytest

import inputs
import oracle
from oracle import adjoint as oadj

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
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _case(name):
    """Small workloads that exercise every path of the adjoint: Helfrich
    with tension, area and volume penalties in duct and Couette flow, and a
    Cahn-Hilliard droplet with the volume penalty."""
    if name == "ch_duct":
        w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.0, u_max=0.05, dt=0.01)
        w.k_vol = 0.002
        dt = 0.01
    else:
        kind = inputs.COUETTE if name == "helfrich_couette" else inputs.POISEUILLE_DUCT
        nz = 8 if name == "helfrich_couette" else 12
        w = inputs.vesicle(16, 12, nz, kind, 0.85, 1.0, dt=5e-4, b_range=(0.25, 0.3),
                           u_max=0.2, v_wall=0.2)
        w.k_area, w.k_vol, w.sigma, w.kappa = 0.4, 0.02, 0.3, 1.3
        dt = 5e-4
    rng = np.random.default_rng(3)
    target = w.phi0 + 0.05 * rng.standard_normal(w.phi0.shape)
    return w, dt, target


def _tape(V, w, prec, every, tol=None):
    from paper_2601_05031_gb300.adjoint import Tape
    t = Tape.from_workload(w, V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED, every=every,
                           tol=1e-12 if prec == "fp64" else 1e-11)
    sp = t.sim.solver_params()
    sp.tol = 1e-13 if prec == "fp64" else 1e-11
    V.vsv_set_solver(t.sim.g, sp)
    return t


def _gpu_gradient(V, w, dt, target, N, prec, every):
    import torch
    t = _tape(V, w, prec, every)
    phiN = t.forward(torch.from_numpy(w.phi0), N, dt)
    pb = w.h ** 3 * (phiN - torch.from_numpy(target).to(phiN.device))
    J = 0.5 * float(torch.sum(pb * (phiN - torch.from_numpy(target).to(phiN.device))))
    g0, dk, ds = t.backward(pb)
    info = t.info()
    out = (J, g0.cpu().numpy(), dk, ds, phiN.cpu().numpy(), t.sim.field(V.VSV_FIELD_PHI), info)
    t.close()
    return out


@pytest.mark.parametrize("case", ["helfrich_duct", "helfrich_couette", "ch_duct"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gradient_vs_oracle_adjoint(V, case, prec):
    """dJ/dphi^0, dJ/dkappa, dJ/dsigma of 5 steps with checkpoints every 2
    steps (three segments, the last one ragged) against the oracle."""
    w, dt, target = _case(case)
    N = 5
    p = oracle.params_from_workload(w)
    Jo, go, ko, so = oadj.gradient(p, w.phi0, dt, N, target)
    J, g, k, s, phiN, phi_after, info = _gpu_gradient(V, w, dt, target, N, prec, 2)
    lim = 1e-9 if prec == "fp64" else 1e-6
    print(case, prec, "J", J, Jo, "phi0bar", rel(g, go), "kappa", k, ko, "sigma", s, so, info)
    assert abs(J - Jo) <= lim * Jo
    assert rel(g, go) < lim, rel(g, go)
    if w.fe_kind == inputs.HELFRICH:
        assert abs(k - ko) <= lim * abs(ko), (k, ko)
    assert abs(s - so) <= lim * abs(so), (s, so)
    assert info["checkpoints"] == 4 and info["recomputed_steps"] == N
    # the backward pass leaves the grid at phi^N
    assert np.array_equal(phi_after, phiN)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gradient_independent_of_checkpoint_interval(V, prec):
    """Segments re-run bit for bit from their checkpoints: the gradient is
    the same, to the bit, for every checkpoint interval."""
    w, dt, target = _case("helfrich_duct")
    N = 6
    ref = _gpu_gradient(V, w, dt, target, N, prec, N)
    for every in (1, 4):
        got = _gpu_gradient(V, w, dt, target, N, prec, every)
        assert np.array_equal(got[1], ref[1])
        assert got[2] == ref[2] and got[3] == ref[3]


def test_gradient_vs_central_differences_of_gpu_forward(V):
    """Central differences of the GPU forward map (FP64) with step 1e-4:
    kappa, sigma and a random direction of phi^0 within 1e-4 relative."""
    import torch
    w, dt, target = _case("helfrich_duct")
    N = 6
    J, g, k, s, *_ = _gpu_gradient(V, w, dt, target, N, "fp64", 3)

    def loss(wl, phi0):
        t = _tape(V, wl, "fp64", N)
        phiN = t.forward(torch.from_numpy(phi0), N, dt).cpu().numpy()
        t.close()
        return 0.5 * wl.h ** 3 * float(np.sum((phiN - target) ** 2))

    step = 1e-4
    for name, grad in (("kappa", k), ("sigma", s)):
        v = getattr(w, name)
        lp = loss(dataclasses.replace(w, **{name: v + step}), w.phi0)
        lm = loss(dataclasses.replace(w, **{name: v - step}), w.phi0)
        fd = (lp - lm) / (2 * step)
        print(name, fd, grad)
        assert abs(fd - grad) <= 1e-4 * abs(fd), (name, fd, grad)
    d = np.random.default_rng(8).standard_normal(w.phi0.shape)
    fd = (loss(w, w.phi0 + step * d) - loss(w, w.phi0 - step * d)) / (2 * step)
    print("phi0 direction", fd, float(np.sum(g * d)))
    assert abs(fd - float(np.sum(g * d))) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fixed_cycle_adjoint_solves(V, prec):
    """Adjoint solves with a fixed number of cycles from the previous reverse
    step's solution (no host synchronisation) stay close to the converged
    gradient, and run exactly that many cycles."""
    import torch
    w, dt, target = _case("helfrich_duct")
    N = 6
    ref = _gpu_gradient(V, w, dt, target, N, prec, 3)
    errs = {}
    for fixed in (2, 4):
        t = _tape(V, w, prec, 3)
        t.set_cycles(fixed)
        phiN = t.forward(torch.from_numpy(w.phi0), N, dt)
        pb = w.h ** 3 * (phiN - torch.from_numpy(target).to(phiN.device))
        g0, dk, ds = t.backward(pb)
        assert t.info()["adjoint_cycles"] == 2 * fixed * (N + 1)
        errs[fixed] = (rel(g0.cpu().numpy(), ref[1]), abs(dk - ref[2]) / abs(ref[2]),
                       abs(ds - ref[3]) / abs(ref[3]))
        t.close()
    print(prec, errs)
    # measured in FP64: 4 cycles 4e-6, 2 cycles 6e-4 (dJ/dsigma, the most
    # sensitive of the three); more cycles, smaller differences
    assert max(errs[4]) < 2e-5, errs
    assert max(errs[2]) < 2e-3, errs
    assert all(a < b for a, b in zip(errs[4], errs[2])), errs


def test_autograd_function_matches_tape(V):
    """The torch.autograd.Function returns the tape's gradients for a loss
    written in torch."""
    import torch
    from paper_2601_05031_gb300.adjoint import trajectory
    w, dt, target = _case("helfrich_duct")
    N = 4
    J, g, k, s, *_ = _gpu_gradient(V, w, dt, target, N, "fp64", 2)
    t = _tape(V, w, "fp64", 2)
    phi0 = torch.from_numpy(w.phi0).cuda().requires_grad_(True)
    kap = torch.tensor(w.kappa, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(w.sigma, dtype=torch.float64, requires_grad=True)
    phiN = trajectory(phi0, kap, sig, t, N, dt)
    tgt = torch.from_numpy(target).cuda()
    loss = 0.5 * w.h ** 3 * torch.sum((phiN - tgt) ** 2)
    loss.backward()
    assert abs(float(loss) - J) <= 1e-14 * J
    assert np.array_equal(phi0.grad.cpu().numpy(), g)
    assert float(kap.grad) == k and float(sig.grad) == s
    t.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inertial_gradient_vs_oracle_adjoint(V, prec):
    """Inertial variant (backward-Euler vorticity, s = rho / (eta dt) = 3):
    the vorticity adjoint is carried between steps through the shifted
    solve; gradients against the oracle."""
    w, dt, target = _case("helfrich_duct")
    w.rho = 3.0 * w.eta * dt
    N = 5
    p = oracle.params_from_workload(w)
    Jo, go, ko, so = oadj.gradient(p, w.phi0, dt, N, target)
    J, g, k, s, phiN, phi_after, info = _gpu_gradient(V, w, dt, target, N, prec, 2)
    lim = 1e-9 if prec == "fp64" else 1e-6
    print("inertial", prec, "phi0bar", rel(g, go), "kappa", k, ko, "sigma", s, so)
    assert abs(J - Jo) <= lim * Jo
    assert rel(g, go) < lim, rel(g, go)
    assert abs(k - ko) <= lim * abs(ko), (k, ko)
    assert abs(s - so) <= lim * abs(so), (s, so)
    # the inertial term changes the gradient by far more than the bar
    p.rho = 0.0
    _, go0, ko0, _ = oadj.gradient(p, w.phi0, dt, N, target)
    assert abs(ko0 - ko) > 100 * lim * abs(ko)


def test_fit_module_small(V):
    """The fitting run end to end on a small grid: central differences of
    the mixed forward map agree with the adjoint within 1e-4 relative, and
    Adam lowers the loss."""
    from paper_2601_05031_gb300 import fit
    res = fit.run(nx=64, ny=32, nz=32, nsteps=20, every=5, adam_steps=4)
    fd = res["finite_differences"]
    print({k: v["rel_err"] for k, v in fd.items() if isinstance(v, dict)})
    for name in ("kappa", "sigma", "phi0_direction"):
        assert fd[name]["rel_err"] < 1e-4, (name, fd[name])
    assert res["fit"]["final"]["loss"] < res["start"]["loss"]
    assert res["tape"]["checkpoints"] == 5 and res["tape"]["recomputed_steps"] == 20
    assert res["adjoint_kernels"]["launches"] > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tape_over_caller_owned_memory(V, prec):
    """A tape whose device memory is the caller's (vsv_tape_create_in, as
    adjoint.Tape uses it) gives the gradient of a library-allocated tape
    (vsv_tape_create) bit for bit; it allocates no device memory of its own,
    rejects a forward pass longer than it was sized for (nothing run), and
    refuses too small, misaligned or host workspaces."""
    import ctypes
    import torch
    from paper_2601_05031_gb300.sim import Simulation
    w, dt, target = _case("helfrich_duct")
    N, every = 5, 2
    p = V.VSV_FP64 if prec == "fp64" else V.VSV_MIXED
    res = []
    for owned in (False, True):
        sim = Simulation.from_workload(w, p)
        sp = sim.solver_params()
        sp.tol = 1e-13 if prec == "fp64" else 1e-11
        V.vsv_set_solver(sim.g, sp)
        nb = V.vsv_tape_workspace_bytes(sim.g, every, N)
        phi0 = torch.from_numpy(w.phi0).to(sim.device).contiguous()
        tgt = torch.from_numpy(target).to(sim.device)
        g0 = torch.empty_like(phi0)
        drops = []
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        if owned:
            ws = torch.empty(nb, dtype=torch.uint8, device=sim.device)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            t = V.vsv_tape_create_in(sim.g, every, N, 0.0, ws.data_ptr(), nb)
        else:
            t = V.vsv_tape_create(sim.g, every, 0.0)
        V.vsv_tape_forward(t, sim.g, phi0.data_ptr(), V.VSV_DTYPE_F64, 1, N, dt)
        torch.cuda.synchronize()
        drops.append(free0 - torch.cuda.mem_get_info()[0])
        phiN = sim.field(V.VSV_FIELD_PHI, torch.float64, on_device=True)
        pb = (w.h ** 3 * (phiN - tgt)).contiguous()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        dk, ds = V.vsv_tape_backward(t, sim.g, pb.data_ptr(), g0.data_ptr(), 1)
        torch.cuda.synchronize()
        drops.append(free1 - torch.cuda.mem_get_info()[0])
        if owned:
            # the library allocated no device memory for the tape's passes
            assert drops == [0, 0], drops
            assert V.vsv_tape_bytes(t) == nb
            # a longer forward pass than the workspace holds: refused, nothing run
            st = V.lib().vsv_tape_forward(t, ctypes.c_void_p(phi0.data_ptr()), V.VSV_DTYPE_F64, 1,
                                          N + every, dt)
            assert st == V.VSV_ENOMEM
        else:
            assert drops[0] > 0, drops   # the allocating tape's checkpoints
        res.append((g0.cpu().numpy(), dk, ds))
        V.vsv_tape_destroy(t)
        if owned:
            # bad workspaces
            assert V.vsv_tape_create_in(sim.g, every, N, 0.0, ws.data_ptr(), nb - 1,
                                        check=False)[1] == V.VSV_ENOMEM
            assert V.vsv_tape_create_in(sim.g, every, N, 0.0, ws.data_ptr() + 16, nb - 256,
                                        check=False)[1] == V.VSV_EINVAL
            host = np.zeros(nb + 256, dtype=np.uint8)
            hp = (host.ctypes.data + 255) // 256 * 256
            assert V.vsv_tape_create_in(sim.g, every, N, 0.0, hp, nb, check=False)[1] == V.VSV_EINVAL
            assert V.vsv_tape_create_in(sim.g, 0, N, 0.0, ws.data_ptr(), nb,
                                        check=False)[1] == V.VSV_EINVAL
            del ws
        sim.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]
    assert np.any(res[0][0] != 0)
