"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, eigenvectors, exact identities, the paper's worked constants
(tests/golden/closed_forms.json) or an independently written loop
transcription.  No GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import inputs
import oracle
from oracle import brute
from oracle.flow import base_flow, body_free_fields, duct_profile
from oracle.grid import pad_mirror, lap, grad, curl, pad_flow
from oracle.poisson import (apply_poisson, poisson_matrix, solve_poisson,
                            solve_poisson_dense, solve_flow_component)
from oracle.free_energy import (chem_potential, helfrich_energy, ch_energy, area, volume,
                                prefactor_cf)
from oracle.step import OracleParams, init_state, step, velocity, vorticity_source, phi_rate

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _params(nx, ny, nz, flow_kind=inputs.QUIESCENT, fe_kind=inputs.CAHN_HILLIARD, **kw):
    base = dict(nx=nx, ny=ny, nz=nz, h=1.0, flow_kind=flow_kind, u_max=0.0, v_lo=0.0,
                v_hi=0.0, eta=1.0, fe_kind=fe_kind, sigma=1.0, kappa=1.0, eps=1.0,
                mobility=1.0, k_area=0.0, k_vol=0.0)
    base.update(kw)
    return OracleParams(**base)


# ------------------------------------------------------------ Poisson (C-P1, C-P2)
@pytest.mark.parametrize("periodic", [(True, False, False), (True, False, True),
                                      (False, False, False), (True, True, False)])
def test_sin_product_eigenvector(periodic):
    """Manufactured sin/cos products are exact eigenvectors of the 7-point
    operator with zero data on the ghost nodes (Dirichlet) or wrap."""
    nz, ny, nx, h = 6, 5, 8, 0.7
    kx, ky, kz = 2, 3, 1
    lam = 0.0
    facs = []
    for n, per, kk in ((nx, periodic[0], kx), (ny, periodic[1], ky), (nz, periodic[2], kz)):
        j = np.arange(n)
        if per:
            th = 2 * math.pi * kk / n
            facs.append(np.cos(th * j + 0.3))
        else:
            th = math.pi * kk / (n + 1)
            facs.append(np.sin(th * (j + 1)))
        lam += (2 * math.cos(th) - 2) / h ** 2
    u = facs[2][:, None, None] * facs[1][None, :, None] * facs[0][None, None, :]
    Lu = apply_poisson(u, h, periodic)
    assert np.max(np.abs(Lu - lam * u)) < 1e-12
    for solver in (solve_poisson, solve_poisson_dense):
        x = solver(lam * u, h, periodic)
        assert np.max(np.abs(x - u)) < 1e-12


def test_mirror_laplacian_cosine_eigenvector():
    """Face-mirror (no-flux) ghosts: cos(pi k (j + 1/2) / n) is an exact
    eigenvector with eigenvalue 2 cos(pi k / n) - 2."""
    nz, ny, nx = 7, 6, 5
    ky, kz, kx = 2, 3, 1
    y = np.cos(math.pi * ky * (np.arange(ny) + 0.5) / ny)
    z = np.cos(math.pi * kz * (np.arange(nz) + 0.5) / nz)
    x = np.cos(2 * math.pi * kx * np.arange(nx) / nx)
    u = z[:, None, None] * y[None, :, None] * x[None, None, :]
    lam = sum(2 * math.cos(t) - 2 for t in (math.pi * ky / ny, math.pi * kz / nz,
                                             2 * math.pi * kx / nx))
    L = lap(pad_mirror(u, 1, False), 1.0)
    assert np.max(np.abs(L - lam * u)) < 1e-13


@pytest.mark.parametrize("periodic", [(True, False, False), (True, False, True),
                                      (False, True, False)])
def test_spectral_matches_sparse_direct(periodic):
    b = inputs.random_field((5, 6, 7), seed=3)
    x1 = solve_poisson(b, 0.5, periodic)
    x2 = solve_poisson_dense(b, 0.5, periodic)
    assert np.max(np.abs(x1 - x2)) / np.max(np.abs(x2)) < 1e-12
    r = apply_poisson(x1, 0.5, periodic) - b
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(b)) * 16


def test_matrix_equals_stencil_and_loops():
    """The assembled matrix equals the stencil form and a loop-assembled
    dense matrix (wall data zero)."""
    p = _params(4, 3, 5, flow_kind=inputs.POISEUILLE_DUCT)
    x = inputs.random_field((5, 3, 4), seed=1)
    L = poisson_matrix(x.shape, 1.0, (True, False, False))
    y1 = (L @ x.reshape(-1)).reshape(x.shape)
    y2 = apply_poisson(x, 1.0, (True, False, False))
    assert np.max(np.abs(y1 - y2)) < 1e-13
    ring = np.zeros((7, 5))
    xb = brute._dense_solve(y2, ring, p)
    assert np.max(np.abs(xb - x)) < 1e-11


# ------------------------------------------------------------ inertial variant (SM eq. 36)
def _eigvec(shape, h, periodic, ks, phase=0.3):
    """Sin/cos-product eigenvector of the 7-point operator and its eigenvalue
    (Dirichlet data on the ghost nodes, or wrap)."""
    nz, ny, nx = shape
    lam = 0.0
    facs = []
    for n, per, kk in ((nx, periodic[0], ks[0]), (ny, periodic[1], ks[1]), (nz, periodic[2], ks[2])):
        j = np.arange(n)
        if per:
            th = 2 * math.pi * kk / n
            facs.append(np.cos(th * j + phase))
        else:
            th = math.pi * kk / (n + 1)
            facs.append(np.sin(th * (j + 1)))
        lam += (2 * math.cos(th) - 2) / h ** 2
    return facs[2][:, None, None] * facs[1][None, :, None] * facs[0][None, None, :], lam


@pytest.mark.parametrize("periodic", [(True, False, False), (True, False, True), (True, True, True)])
def test_shifted_eigenvector(periodic):
    """(L_h - s) u = (lambda - s) u for the product eigenvectors; both exact
    solvers invert the shifted operator, also with every axis periodic."""
    shape, h, s = (6, 5, 8), 0.7, 3.7
    u, lam = _eigvec(shape, h, periodic, (2, 1, 1))
    Lu = apply_poisson(u, h, periodic) - s * u
    assert np.max(np.abs(Lu - (lam - s) * u)) < 1e-12
    for solver in (solve_poisson, solve_poisson_dense):
        x = solver((lam - s) * u, h, periodic, s)
        assert np.max(np.abs(x - u)) < 1e-12


def test_inertial_vorticity_decays_as_backward_euler():
    """No body, walls at rest: one backward-Euler step of SM eq. 36 maps a
    vorticity eigenmode to s / (s - lambda) times itself (s = rho / (eta dt)),
    and the stream vector follows as psi = -omega / lambda."""
    nx, ny, nz = 8, 7, 6
    p = _params(nx, ny, nz, flow_kind=inputs.QUIESCENT, eta=0.7, rho=2.0)
    st = init_state(p, _no_body(nx, ny, nz))
    u, lam = _eigvec((nz, ny, nx), 1.0, (True, False, False), (1, 2, 1))
    amp = (0.3, -0.1, 0.2)
    st.omega = [a * u for a in amp]
    dt = 0.05
    s = p.rho / (p.eta * dt)
    g = s / (s - lam)
    assert 0.0 < g < 1.0
    for k in range(1, 4):
        step(st, dt)
        assert np.max(np.abs(st.phi - 1.0)) == 0.0
        for c in range(3):
            w = amp[c] * g ** k * u
            assert np.max(np.abs(st.omega[c] - w)) < 1e-13
            assert np.max(np.abs(st.psi[c] + w / lam)) < 1e-12


def test_inertial_step_tends_to_stokes_linearly_in_density():
    """As rho -> 0 the inertial step tends to the non-inertial one (eq.
    gen1): the difference in omega is proportional to rho."""
    w = inputs.droplet_duct(nx=12, ny=8, nz=8, radius=2.5, dt=0.01)
    base = dict(nx=w.nx, ny=w.ny, nz=w.nz, h=1.0, flow_kind=w.flow_kind, u_max=w.u_max,
                v_lo=0.0, v_hi=0.0, eta=w.eta, fe_kind=w.fe_kind, sigma=w.sigma, kappa=0.0,
                eps=w.eps, mobility=1.0, k_area=0.0, k_vol=0.0)
    om = {}
    for rho in (0.0, 1e-6, 2e-6):
        st = init_state(OracleParams(**base, rho=rho), w.phi0)
        st.omega = [o * 0.5 for o in st.omega]   # start away from the Stokes vorticity
        step(st, w.dt)
        om[rho] = np.stack(st.omega)
    d1 = np.max(np.abs(om[1e-6] - om[0.0]))
    d2 = np.max(np.abs(om[2e-6] - om[0.0]))
    assert d1 > 0.0
    assert abs(d2 / d1 - 2.0) < 1e-3


# ------------------------------------------------------------ base flows (C-P3..5)
def _no_body(nx, ny, nz):
    return np.ones((nz, ny, nx))


def test_couette_body_free_is_exact():
    """With no body the discrete Couette flow is the closed form: psi_z
    quadratic, omega_z constant, v_x linear from v_lo to v_hi (walls on the
    ghost nodes, y = (j + 1) h, H = (ny + 1) h)."""
    nx, ny, nz, vlo, vhi = 6, 9, 4, -0.05, 0.05
    p = _params(nx, ny, nz, flow_kind=inputs.COUETTE, v_lo=vlo, v_hi=vhi, eta=0.3)
    st = init_state(p, _no_body(nx, ny, nz))
    H = ny + 1.0
    y = np.arange(ny) + 1.0
    psi_z = vlo * y + (vhi - vlo) * y ** 2 / (2 * H)
    assert np.max(np.abs(st.psi[2] - psi_z[None, :, None])) < 1e-13
    assert np.max(np.abs(st.omega[2] + (vhi - vlo) / H)) < 1e-15
    for c in (0, 1):
        assert np.max(np.abs(st.psi[c])) < 1e-15 and np.max(np.abs(st.omega[c])) < 1e-15
    v = velocity(st)
    assert np.max(np.abs(v[0] - (vlo + (vhi - vlo) * y / H)[None, :, None])) < 1e-14
    assert abs(GOLD["couette_vorticity_vw0p05_H257"]["value"] - (-(0.1) / 257)) < 1e-18
    phi_before = st.phi.copy()
    step(st, 0.01)
    assert np.max(np.abs(st.phi - phi_before)) == 0.0
    assert np.max(np.abs(st.psi[2] - psi_z[None, :, None])) < 1e-13


def test_planar_poiseuille_closed_form():
    """Planar Poiseuille: psi_z cubic and omega_z linear are exact discrete
    solutions; the central-difference velocity is v_x - (4/3) U h^2 / H^2."""
    nx, ny, nz, U = 4, 11, 3, 0.07
    p = _params(nx, ny, nz, flow_kind=inputs.POISEUILLE_PLANAR, u_max=U)
    st = init_state(p, _no_body(nx, ny, nz))
    H = ny + 1.0
    y = np.arange(ny) + 1.0
    psi_z = 4 * U * (H * y ** 2 / 2 - y ** 3 / 3) / H ** 2
    om_z = -4 * U * (H - 2 * y) / H ** 2
    assert np.max(np.abs(st.psi[2] - psi_z[None, :, None])) < 1e-13
    assert np.max(np.abs(st.omega[2] - om_z[None, :, None])) < 1e-14
    v = velocity(st)
    vx = 4 * U * y * (H - y) / H ** 2 - 4.0 / 3.0 * U / H ** 2
    assert np.max(np.abs(v[0] - vx[None, :, None])) < 1e-14


def _duct_series(y, z, a, b, G=1.0, terms=60):
    """Textbook rectangular-duct Poiseuille solution of -lap u = G,
    u = 0 on the walls of [0, a] x [0, b] (single cosh series)."""
    u = 0.5 * G * y * (a - y)
    for m in range(1, 2 * terms, 2):
        u = u - (4 * G * a * a / (math.pi ** 3 * m ** 3)) * (
            np.cosh(m * math.pi * (z - b / 2) / a) / math.cosh(m * math.pi * b / (2 * a))
        ) * np.sin(m * math.pi * y / a)
    return u


def test_duct_converges_second_order():
    """Body-free duct velocity converges at second order to the series
    solution (same physical duct, spacing halved)."""
    errs = []
    for n, h in ((31, 0.5), (63, 0.25)):
        p = _params(2, n, n, flow_kind=inputs.POISEUILLE_DUCT, u_max=0.05, h=h)
        st = init_state(p, _no_body(2, n, n))
        vx = velocity(st)[0][:, :, 0]          # [k][j]
        H = (n + 1) * h
        c = (np.arange(n) + 1.0) * h
        Z, Y = np.meshgrid(c, c, indexing="ij")
        ref = _duct_series(Y, Z, H, H)
        ref *= 0.05 / _duct_series(np.array(H / 2), np.array(H / 2), H, H)
        errs.append(np.max(np.abs(vx - ref)))
        assert np.max(np.abs(velocity(st)[1])) < 1e-15 and np.max(np.abs(velocity(st)[2])) < 1e-15
    assert errs[0] < 3e-4
    rate = math.log2(errs[0] / errs[1])
    assert 1.75 < rate < 2.3, (errs, rate)


def test_duct_profile_is_discrete_poisson_solution():
    u0, chi = duct_profile(7, 5, 1.0, 0.05)
    assert abs(u0.max() - 0.05) < 1e-16
    Lu = lap(pad_flow(u0[:, :, None], np.zeros((7, 9)), False), 1.0)[:, :, 0]
    ratio = Lu / Lu.mean()
    assert np.max(np.abs(ratio - 1)) < 1e-12 and Lu.mean() < 0


def test_div_curl_vanishes():
    """Central differences commute: div(curl psi) = 0 to round-off for any
    psi and any wall data (C-P6)."""
    nz, ny, nx = 5, 6, 7
    psi = [inputs.random_field((nz, ny, nx), seed=s) for s in range(3)]
    rng = np.random.default_rng(9)
    ghosts = [rng.standard_normal((nz + 2, ny + 2)) for _ in range(3)]
    v = curl(psi, ghosts, 1.0, False)
    # divergence needs v on the wall nodes: use an extended field where the
    # curl is taken on a grid one node larger (walls become interior)
    big = [np.zeros((nz + 2, ny + 2, nx)) for _ in range(3)]
    for c in range(3):
        big[c][1:-1, 1:-1, :] = psi[c]
        big[c][0, :, :] = ghosts[c][0][:, None]
        big[c][-1, :, :] = ghosts[c][-1][:, None]
        big[c][:, 0, :] = ghosts[c][:, 0][:, None]
        big[c][:, -1, :] = ghosts[c][:, -1][:, None]
    outer = [np.zeros((nz + 4, ny + 4)) for _ in range(3)]
    vb = curl(big, outer, 1.0, False)
    dv = grad(np.pad(vb[0], ((1, 1), (1, 1), (1, 1)), mode="wrap"), 1.0)[0] \
        + grad(np.pad(vb[1], ((1, 1), (1, 1), (1, 1)), mode="wrap"), 1.0)[1] \
        + grad(np.pad(vb[2], ((1, 1), (1, 1), (1, 1)), mode="wrap"), 1.0)[2]
    inner = dv[2:-2, 2:-2, :]
    assert np.max(np.abs(inner)) < 1e-13
    for c in range(3):  # the interior curl equals the padded-grid curl there
        assert np.max(np.abs(vb[c][1:-1, 1:-1, :] - v[c])) < 1e-14


# ------------------------------------------------------------ chemical potential (C-P7..10)
@pytest.mark.parametrize("fe_kind,zper,sigma", [(inputs.CAHN_HILLIARD, False, 0.7),
                                                (inputs.HELFRICH, False, 0.0),
                                                (inputs.HELFRICH, True, 0.0),
                                                (inputs.HELFRICH, False, 0.7),
                                                (inputs.HELFRICH, True, 0.4)])
def test_energy_gradient_identity(fe_kind, zper, sigma):
    """mu_i = h^-3 dF_h/dphi_i exactly (symmetric mirror / periodic
    Laplacian), checked by central finite differences of the discrete
    energy; fixes the prefactor 2 C_F, the signs and the wall treatment.
    Helfrich with sigma != 0: F = C_F h^3 sum g^2 + sigma A_f, the area of
    SM eq. 32 with face differences, 3 / (2 sqrt 2) h^3 sum [(phi^2 - 1)^2 /
    (4 eps) + eps / 2 |D+ phi|^2]."""
    nz, ny, nx, h = 4, 5, 3, 0.8
    rng = np.random.default_rng(4)
    phi = 0.6 * rng.standard_normal((nz, ny, nx))
    kappa, eps = 1.3, 1.1
    mu = chem_potential(phi, fe_kind, h, zper, sigma=sigma, kappa=kappa, eps=eps)
    if fe_kind == inputs.HELFRICH:
        def area_f(ph):
            bulk = np.sum((ph * ph - 1.0) ** 2) / (4.0 * eps)
            faces = np.sum((np.roll(ph, -1, axis=2) - ph) ** 2)
            faces += np.sum((ph[:, 1:] - ph[:, :-1]) ** 2)
            faces += np.sum((np.roll(ph, -1, axis=0) - ph) ** 2 if zper else (ph[1:] - ph[:-1]) ** 2)
            return 3.0 / (2.0 * math.sqrt(2.0)) * h ** 3 * (bulk + 0.5 * eps * faces / h ** 2)
        F = lambda ph: helfrich_energy(ph, kappa, eps, h, zper) + sigma * area_f(ph)
    else:
        F = lambda ph: ch_energy(ph, sigma, h, zper)
    d = 1e-5
    for (k, j, i) in [(0, 0, 0), (1, 2, 1), (3, 4, 2), (2, 0, 1), (0, 4, 0)]:
        pp, pm = phi.copy(), phi.copy()
        pp[k, j, i] += d
        pm[k, j, i] -= d
        fd = (F(pp) - F(pm)) / (2 * d) / h ** 3
        assert abs(fd - mu[k, j, i]) < 1e-7 * max(1.0, abs(mu[k, j, i])), (k, j, i, fd, mu[k, j, i])


def _sphere(n, h, R, eps):
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((X - n * h / 2) ** 2 + (Y - n * h / 2) ** 2 + (Z - n * h / 2) ** 2)
    return np.tanh((r - R) / (math.sqrt(2) * eps)), r


def test_sphere_area_and_helfrich_energy():
    """tanh sphere: A_h -> 4 pi R^2 (SM eq. 32 normalisation) and the
    phase-field bending energy -> 8 pi kappa (eq. 30 normalisation)."""
    eps, R = 1.0, 8.0
    res = []
    for h in (0.5, 0.25):
        n = int(round(2 * (R + 6 * eps) / h))
        phi, _ = _sphere(n, h, R, eps)
        res.append((area(phi, eps, h, False) / (4 * math.pi * R * R),
                    helfrich_energy(phi, 1.0, eps, h, False) / GOLD["helfrich_sphere_energy_kappa1"]["value"]))
    # both within a few percent and improving under refinement
    for a, f in res:
        assert abs(a - 1) < 0.03 and abs(f - 1) < 0.05, res
    assert abs(res[1][1] - 1) <= abs(res[0][1] - 1) + 1e-3


def test_flat_interface_is_stationary_at_second_order():
    """Flat CH profile tanh(z / sqrt(2 sigma)) (SM eq. 10, sigma = eps^2):
    mu = O(h^2)."""
    errs = []
    for h in (0.5, 0.25):
        ny = int(round(24 / h))
        y = (np.arange(ny) + 1.0) * h
        prof = np.tanh((y - (ny + 1) * h / 2) / math.sqrt(2.0))
        phi = np.broadcast_to(prof[None, :, None], (3, ny, 2)).copy()
        mu = chem_potential(phi, inputs.CAHN_HILLIARD, h, True, sigma=1.0)
        errs.append(np.max(np.abs(mu)))
    rate = math.log2(errs[0] / errs[1])
    assert errs[0] < 0.02 and 1.8 < rate < 2.2, (errs, rate)


def test_gibbs_thomson_and_laplace_jump():
    """CH tanh sphere: the interface-weighted mu equals -gamma / R with
    gamma = 2 sqrt(2 sigma)/3 (SM eqs. 13-15; phi = -1 inside so mu < 0),
    and int mu dphi = [phi] mu = 2 gamma / R in magnitude (Laplace jump,
    SM eqs. 19, 25)."""
    gamma = GOLD["surface_tension_sigma1"]["value"]
    assert abs(inputs.surface_tension(1.0) - gamma) < 1e-15
    R, h, eps = 12.0, 0.5, 1.0
    n = int(round(2 * (R + 7) / h))
    phi, r = _sphere(n, h, R, eps)
    mu = chem_potential(phi, inputs.CAHN_HILLIARD, h, False, sigma=1.0)
    gx, gy, gz = grad(pad_mirror(phi, 1, False), h)
    # radial derivative of phi (positive outward)
    c = n * h / 2
    Z, Y, X = np.meshgrid(*(3 * [(np.arange(n) + 0.5) * h]), indexing="ij")
    dr = (gx * (X - c) + gy * (Y - c) + gz * (Z - c)) / np.maximum(r, 1e-12)
    shell = np.abs(r - R) < 6
    w = dr * (r / R) ** -2          # per-unit-area weights on the shell
    proj = float(np.sum(mu[shell] * w[shell]) / np.sum(w[shell]))
    assert abs(proj / (-gamma / R) - 1) < 0.05, proj
    jump = float(np.sum(mu[shell] * w[shell]) * h ** 3 / (4 * math.pi * R * R))
    assert abs(abs(jump) / (2 * gamma / R) - 1) < 0.05, jump
    assert GOLD["phi_jump_integral"]["value"] == 2.0


def test_profile_gradient_integral():
    """int (d phi0/dz)^2 dz = 2 sqrt 2 / (3 sqrt sigma) (SM eqs. 14-15)."""
    for sig, key in ((1.0, "profile_gradient_integral_sigma1"),
                     (2.25, "profile_gradient_integral_sigma2p25")):
        z = np.linspace(-40, 40, 400001)
        d = 1.0 / (np.cosh(z / math.sqrt(2 * sig)) ** 2 * math.sqrt(2 * sig))
        val = float(np.sum(d * d) * (z[1] - z[0]))
        assert abs(val - GOLD[key]["value"]) < 1e-6


def test_reduced_volume_and_input_geometry():
    assert abs(inputs.reduced_volume(5.0, 5.0) - GOLD["reduced_volume_sphere"]["value"]) < 1e-12
    for vr in (0.7, 0.8, 0.9, 0.98):
        a = inputs.prolate_axis_for(vr, 10.0)
        assert abs(inputs.reduced_volume(a, 10.0) - vr) < 1e-10 and a > 10.0


# ------------------------------------------------------------ dynamics
def test_advection_of_sine_closed_form():
    """phi = A sin(2 pi x / Lx) in body-free Couette, M = 0: grad phi x grad
    mu = 0 so the flow is the base flow, and one step is
    phi - dt v_x(y) A sin(k h)/h cos(k x) (eq. gen2 sign, central D)."""
    nx, ny, nz, A, dt = 16, 7, 3, 0.3, 0.5
    p = _params(nx, ny, nz, flow_kind=inputs.COUETTE, v_lo=-0.2, v_hi=0.3, mobility=0.0)
    k = 2 * math.pi / nx
    x = np.arange(nx) * 1.0
    phi0 = np.broadcast_to(A * np.sin(k * x)[None, None, :], (nz, ny, nx)).copy()
    st = init_state(p, phi0)
    for c in range(3):
        assert np.max(np.abs(st.omega[c] - init_state(p, np.ones_like(phi0)).omega[c])) < 1e-14
    H = ny + 1.0
    y = np.arange(ny) + 1.0
    vx = (-0.2 + 0.5 * y / H)[None, :, None]
    expect = phi0 - dt * vx * A * math.sin(k) * np.cos(k * x)[None, None, :]
    step(st, dt)
    assert np.max(np.abs(st.phi - expect)) < 1e-14


def test_source_cross_product_closed_form():
    """f = grad phi x grad mu / eta with phi(x), mu(y): only f_z =
    phi_x mu_y / eta is non-zero (eq. gen1)."""
    nx, ny, nz, eta = 12, 10, 3, 0.4
    p = _params(nx, ny, nz, eta=eta)
    k = 2 * math.pi / nx
    x = np.arange(nx) * 1.0
    yy = np.arange(ny) + 0.5
    phi = np.broadcast_to(np.sin(k * x)[None, None, :], (nz, ny, nx)).copy()
    q = math.pi / ny
    mu = np.broadcast_to(np.cos(q * yy)[None, :, None], (nz, ny, nx)).copy()
    f = vorticity_source(phi, mu, p)
    assert np.max(np.abs(f[0])) < 1e-15 and np.max(np.abs(f[1])) < 1e-15
    px = math.sin(k) * np.cos(k * x)
    my = -math.sin(q) * np.sin(q * yy)
    expect = (my[:, None] * px[None, :]) / eta
    assert np.max(np.abs(f[2][:, 1:-1, :] - expect[None, 1:-1, :])) < 1e-14


def test_volume_penalty_restores_volume():
    """SM eqs. 37-38 reading: lambda_V = K_V (V - V0) > 0 when the body is
    too large, and the next step moves V back toward V0 (C-P11)."""
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.0, u_max=0.0,
                            flow_kind=inputs.QUIESCENT)
    p = oracle.params_from_workload(w)
    p.k_vol = inputs.stable_k_vol(0.01, 1.0, w.ncells, 1.0, 0.5)
    st = init_state(p, w.phi0)
    st.V0 = st.V - 5.0          # body is 5 units too large
    v_before = st.V
    step(st, 0.01)
    assert st.lambda_v > 0
    assert abs(st.V - st.V0) < abs(v_before - st.V0) * 0.9


def test_mass_conservation_of_model_b():
    """Without the volume multiplier, Model-B diffusion and divergence-free
    advection keep sum(phi) constant up to the advection term; with zero
    flow it is exact (no-flux mirror walls)."""
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5, u_max=0.0,
                            flow_kind=inputs.QUIESCENT)
    p = oracle.params_from_workload(w)
    st = init_state(p, w.phi0)
    st.psi = [np.zeros_like(st.phi) for _ in range(3)]
    r = phi_rate(st, 0.0)
    assert abs(float(np.sum(r))) < 1e-11


def test_energy_decreases_and_flow_dissipates():
    """Coupling sign of eq. gen1: for a body at rest between quiescent walls,
    the flow lowers the free energy (dF/dt gains -eta int |grad v|^2); with
    the opposite source sign it would raise it."""
    nx, ny, nz = 20, 16, 16
    w = inputs.droplet_duct(nx=nx, ny=ny, nz=nz, radius=4.0, u_max=0.0,
                            flow_kind=inputs.QUIESCENT)
    c = inputs.channel_centre(nx, ny, nz, 1.0, False)
    w.phi0 = inputs.ellipsoid_phi(nx, ny, nz, 1.0, False, c, (6.0, 3.5, 3.5), 1.0)
    p = oracle.params_from_workload(w)
    p.eta = 0.05
    dt = 1e-3
    st = init_state(p, w.phi0)
    F0 = ch_energy(st.phi, p.sigma, 1.0, False)
    r_flow = phi_rate(st, 0.0)
    st_noflow = init_state(p, w.phi0)
    st_noflow.psi = [np.zeros_like(st.phi) for _ in range(3)]
    r_noflow = phi_rate(st_noflow, 0.0)
    dF_flow = (ch_energy(st.phi + dt * r_flow, p.sigma, 1.0, False) - F0) / dt
    dF_noflow = (ch_energy(st.phi + dt * r_noflow, p.sigma, 1.0, False) - F0) / dt
    assert dF_noflow < 0 and dF_flow < dF_noflow
    from oracle.diagnostics import dissipation_of
    D = dissipation_of(velocity(st), st.bf.vel_b, 1.0, p.eta, False)
    ratio = (dF_noflow - dF_flow) / D
    assert 0.7 < ratio < 1.3, ratio


# ------------------------------------------------------------ transcription (C-P12)
@pytest.mark.parametrize("case", ["ch_duct", "helfrich_couette", "helfrich_planar",
                                  "helfrich_tension"])
def test_brute_force_step_matches(case):
    if case == "ch_duct":
        w = inputs.droplet_duct(nx=6, ny=4, nz=5, radius=1.6, u_max=0.05, dt=0.01)
        p = oracle.params_from_workload(w)
        p.k_vol, p.k_area = 0.3, 0.2
    else:
        kind = inputs.POISEUILLE_PLANAR if case == "helfrich_planar" else inputs.COUETTE
        w = inputs.vesicle(8, 5, 4, kind, 0.9, 1.0, dt=1e-3, b_range=(0.3, 0.35))
        p = oracle.params_from_workload(w)
        p.k_area, p.k_vol = 0.3, 0.01
        if case == "helfrich_tension":
            p.sigma = 0.4
    st = init_state(p, w.phi0)
    st.V0 += 0.5
    st.A0 -= 0.3
    bres = brute.brute_step(st.phi, st.mu, st.psi, st.V, st.V0, st.A0, p, st.bf, w.dt)
    step(st, w.dt)
    for a, b in zip([st.phi, st.mu] + st.omega + st.psi,
                    [bres[0], bres[1]] + bres[2] + bres[3]):
        scale = max(1e-300, np.max(np.abs(b)))
        assert np.max(np.abs(a - b)) <= 1e-11 * scale + 1e-15
    assert abs(st.V - bres[4]) < 1e-10 and abs(st.A - bres[5]) < 1e-10


def test_workload_shapes():
    w = inputs.droplet_24x24x48()
    assert (w.nx, w.ny, w.nz) == (48, 24, 24) and w.phi0.shape == (24, 24, 48)
    assert abs(w.eta - 0.1 * GOLD["surface_tension_sigma1"]["value"] / 0.05) < 1e-12
    assert w.phi0.min() < -0.99 and w.phi0.max() > 0.99


# ------------------------------------------------------------ discrete adjoint (f1)
from oracle import adjoint as adj


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


@pytest.mark.parametrize("zper", [False, True])
def test_adjoint_transposes_dot_product(zper):
    """<A u, w> = <u, A^T w> for each transpose against the forward operator
    it transposes: mirror central differences (oracle.grid.grad of the mirror
    padding), the curl of a stream vector with zero wall data
    (oracle.grid.curl), the mirror Laplacian and the Poisson solve."""
    nz, ny, nx, h = 5, 6, 7, 0.9
    rng = np.random.default_rng(11)
    u = rng.standard_normal((nz, ny, nx))
    w = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    Du = grad(pad_mirror(u, 1, zper), h)
    lhs = sum(_dot(Du[a], w[a]) for a in range(3))
    assert abs(lhs - _dot(u, adj.grad_mirror_t(w, h, zper))) < 1e-12 * max(1.0, abs(lhs))
    us = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    zero = [np.zeros((nz + 2, ny + 2)) for _ in range(3)]
    cu = curl(us, zero, h, zper)
    lhs = sum(_dot(cu[c], w[c]) for c in range(3))
    cw = adj.curl_zero(w, h, zper)
    assert abs(lhs - sum(_dot(us[c], cw[c]) for c in range(3))) < 1e-12 * max(1.0, abs(lhs))
    lu = lap(pad_mirror(u, 1, zper), h)
    assert abs(_dot(lu, w[0]) - _dot(u, lap(pad_mirror(w[0], 1, zper), h))) < 1e-11
    per = (True, False, zper)
    a1 = _dot(solve_poisson(u, h, per), w[1])
    assert abs(a1 - _dot(u, solve_poisson(w[1], h, per))) < 1e-11 * max(1.0, abs(a1))


@pytest.mark.parametrize("fe_kind,sigma,gamma", [(inputs.HELFRICH, 0.0, 0.0),
                                                 (inputs.HELFRICH, 0.6, 0.3),
                                                 (inputs.CAHN_HILLIARD, 0.8, 0.0)])
def test_mu_vjp_against_central_differences(fe_kind, sigma, gamma):
    """(d mu / d phi)^T mubar and the parameter sums against central
    differences of oracle.free_energy.chem_potential."""
    nz, ny, nx, h, eps, kappa = 4, 5, 6, 1.0, 1.2, 1.4
    rng = np.random.default_rng(5)
    phi = np.tanh(rng.standard_normal((nz, ny, nx)))
    d = rng.standard_normal((nz, ny, nx))
    mubar = rng.standard_normal((nz, ny, nx))
    p = _params(nx, ny, nz, fe_kind=fe_kind, sigma=sigma, kappa=kappa, eps=eps)
    mu = lambda ph, **kw: chem_potential(ph, fe_kind, h, False, **{**dict(
        sigma=sigma, kappa=kappa, eps=eps, gamma_a=gamma), **kw})
    pb, kb, sb, gb = adj.mu_vjp(phi, gamma, mubar, p)
    t = 1e-6
    fd = _dot(mubar, (mu(phi + t * d) - mu(phi - t * d)) / (2 * t))
    assert abs(fd - _dot(pb, d)) < 1e-7 * max(1.0, abs(fd)), (fd, _dot(pb, d))
    if fe_kind == inputs.HELFRICH:
        fdk = _dot(mubar, (mu(phi, kappa=kappa + t) - mu(phi, kappa=kappa - t)) / (2 * t))
        assert abs(fdk - kb) < 1e-7 * max(1.0, abs(fdk))
        fdg = _dot(mubar, (mu(phi, gamma_a=gamma + t) - mu(phi, gamma_a=gamma - t)) / (2 * t))
        assert abs(fdg - gb) < 1e-7 * max(1.0, abs(fdg))
    fds = _dot(mubar, (mu(phi, sigma=sigma + t) - mu(phi, sigma=sigma - t)) / (2 * t))
    assert abs(fds - sb) < 1e-7 * max(1.0, abs(fds))


def _adjoint_case(case):
    if case == "ch_duct":
        w = inputs.droplet_duct(nx=10, ny=8, nz=8, radius=2.5, u_max=0.05, dt=0.02)
        p = oracle.params_from_workload(w)
        p.k_vol = 0.002
        dt = 0.02
    else:
        kind = inputs.COUETTE if case == "helfrich_couette" else inputs.POISEUILLE_DUCT
        w = inputs.vesicle(12, 8, 8, kind, 0.85, 1.0, dt=2e-3, b_range=(0.3, 0.35),
                           u_max=0.2, v_wall=0.2)
        p = oracle.params_from_workload(w)
        p.k_area, p.k_vol, p.sigma, p.kappa = 0.4, 0.02, 0.3, 1.3
        dt = 2e-3
        if case == "helfrich_inertial":   # backward-Euler vorticity, s = rho / (eta dt) = 3
            p.rho = 3.0 * p.eta * dt
    return w, p, dt


@pytest.mark.parametrize("case", ["helfrich_duct", "helfrich_couette", "ch_duct",
                                  "helfrich_inertial"])
def test_trajectory_gradient_against_central_differences(case):
    """Gradient of J = h^3/2 sum (phi^N - target)^2 after 4 steps with
    respect to kappa, sigma and two random directions of phi^0, against
    central differences of the forward oracle."""
    import dataclasses
    w, p, dt = _adjoint_case(case)
    N = 4
    rng = np.random.default_rng(3)
    target = w.phi0 + 0.05 * rng.standard_normal(w.phi0.shape)

    def J(pp, phi0):
        return adj.forward(pp, phi0, dt, N)[-1]["phi"]

    def loss(pp, phi0):
        return adj.loss(J(pp, phi0), target, pp.h)

    J0, gphi, gk, gs = adj.gradient(p, w.phi0, dt, N, target)
    assert abs(J0 - loss(p, w.phi0)) < 1e-14 * J0
    t = 1e-5
    for name, g in (("kappa", gk), ("sigma", gs)):
        if name == "kappa" and p.fe_kind != inputs.HELFRICH:
            continue
        v = getattr(p, name)
        lp = loss(dataclasses.replace(p, **{name: v + t}), w.phi0)
        lm = loss(dataclasses.replace(p, **{name: v - t}), w.phi0)
        fd = (lp - lm) / (2 * t)
        assert abs(fd - g) < 1e-6 * abs(fd), (name, fd, g)
    for seed in (1, 2):
        d = np.random.default_rng(seed).standard_normal(w.phi0.shape)
        fd = (loss(p, w.phi0 + t * d) - loss(p, w.phi0 - t * d)) / (2 * t)
        assert abs(fd - _dot(gphi, d)) < 1e-6 * abs(fd), (seed, fd, _dot(gphi, d))
