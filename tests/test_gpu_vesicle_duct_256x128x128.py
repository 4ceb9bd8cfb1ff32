"""The single-vesicle duct workload at 256 x 128 x 128 (x the flow axis):
Helfrich vesicle of reduced volume 0.8 with area and volume penalties in
Poiseuille flow, 2000 steps of dt = 1e-4.  The mixed path in the schedule
bench.py times (bench.BENCH_CYCLES fixed V(2,2)-cycles per solve with
over-relaxed smoothing, extrapolated guess) is
compared along the run with the FP64 GPU path solved to a relative residual
of 1e-12 each step; at the end one step is checked cell by cell against the
oracle's operators on sampled windows (the oracle cannot run 2000 steps of
4.2 M cells in a test)."""
import numpy as np
import pytest

import inputs
import oracle
from oracle.grid import lap, pad_mirror, curl, grad
from oracle.free_energy import chem_potential
from test_gpu_fullsize import M, _core, _interior_windows_around_body

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


def test_mixed_against_fp64_over_2000_steps_and_oracle_sample(V):
    import torch
    import bench
    w = inputs.vesicle_poiseuille_256x128x128()
    mixed = bench.make_sim(w, V.VSV_MIXED, bench.BENCH_CYCLES, bench.BENCH_EXTRAPOLATE)
    fp64 = bench.make_sim(w, V.VSV_FP64, 0)
    sp = fp64.solver_params()
    sp.tol = 1e-12
    V.vsv_set_solver(fp64.g, sp)

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    def vel(s):
        return torch.stack([s.field(V.VSV_FIELD_VEL_X + c, np.float64, on_device=True)
                            for c in range(3)])

    done, errs = 0, {}
    for mark in (10, 100, 1000, 2000):
        mixed.step(mark - done, w.dt)
        fp64.step(mark - done, w.dt)
        done = mark
        errs[mark] = (rel(mixed.field(V.VSV_FIELD_PHI, np.float64, on_device=True),
                          fp64.field(V.VSV_FIELD_PHI, np.float64, on_device=True)),
                      rel(vel(mixed), vel(fp64)))
    print("256x128x128 mixed vs FP64 (phi, velocity):", errs)
    # measured on GB300: phi 1.4e-10 .. 2.8e-10, velocity 4.4e-8 .. 3.4e-7
    for mark, (ephi, evel) in errs.items():
        assert ephi <= 1e-6 and evel <= 1e-6, (mark, ephi, evel)
    fp64.close()

    # one more mixed step, checked against the oracle's operators
    p = oracle.params_from_workload(w)
    d0 = mixed.diagnostics()
    phi0 = mixed.field(V.VSV_FIELD_PHI)
    mu0 = mixed.field(V.VSV_FIELD_MU)
    psi0 = [mixed.field(V.VSV_FIELD_PSI_X + c) for c in range(3)]
    mixed.step(1, w.dt)
    d1 = mixed.diagnostics()
    phi1 = mixed.field(V.VSV_FIELD_PHI)
    mu1 = mixed.field(V.VSV_FIELD_MU)
    mixed.close()
    h = w.h
    dphi_err = dphi_ref = mu_err = mu_ref = 0.0
    for win in _interior_windows_around_body(w, 16, 11):
        ghosts = [np.zeros((2 * M + 3, 2 * M + 3))] * 3
        v = curl([ps[win] for ps in psi0], ghosts, h, False)
        gp = grad(pad_mirror(phi0[win], 1, False), h)
        rate = p.mobility * (lap(pad_mirror(mu0[win], 1, False), h) + d0["lambda_v"]) - \
            (v[0] * gp[0] + v[1] * gp[1] + v[2] * gp[2])
        dref = _core(w.dt * rate, 1)
        dphi_err = max(dphi_err, float(np.max(np.abs(_core(phi1[win] - phi0[win], 1) - dref))))
        dphi_ref = max(dphi_ref, float(np.max(np.abs(dref))))
        mref = chem_potential(phi1[win], p.fe_kind, h, False, sigma=p.sigma, kappa=p.kappa,
                              eps=p.eps, gamma_a=d1["gamma_a"])
        mu_err = max(mu_err, float(np.max(np.abs(_core(mu1[win] - mref, 2)))))
        mu_ref = max(mu_ref, float(np.max(np.abs(_core(mref, 2)))))
    print("after 2000 steps, sampled: dphi %.3e of %.3e, mu %.3e of %.3e" %
          (dphi_err, dphi_ref, mu_err, mu_ref))
    # the same bounds as at 512 x 256 x 256
    assert dphi_err <= 2e-6 * dphi_ref, (dphi_err, dphi_ref)
    assert mu_err <= 5e-9 * mu_ref, (mu_err, mu_ref)
