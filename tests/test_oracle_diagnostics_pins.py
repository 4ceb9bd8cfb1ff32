"""Pins of the oracle's observables (oracle/diagnostics.py) against closed forms.

The observables are the in-plane stress of the in-plane-shear section
(sigma_ij = eta (d_j v_i + d_i v_j), sigma_t, the profile <sigma_xy>(y)),
the dissipation and the relative hydrodynamic resistance (D - D0) / D0, the
flow deviations of the results section, the reduced volume (SM eq. 40), the
energies (eq. 30, eq. 31), the centre of mass and the divergences.  Every
expected value below comes from a closed form, a discrete identity of
trigonometric functions or a continuum limit, not from the oracle's own
formulas.  No GPU.

Discrete calculus used for the closed forms: the central difference of
sin(t n) is cos(t n) sin(t) / h and that of cos(t n) is -sin(t n) sin(t) / h
(sum-to-product), exact on a periodic axis whose extent fits whole periods
and on a walled axis whose ghost values follow the same function.
"""
import math

import numpy as np
import pytest

import inputs
from oracle.diagnostics import diagnostics
from oracle.flow import base_flow
from oracle.step import OracleParams, OracleState, init_state


def _params(nx, ny, nz, flow_kind=inputs.QUIESCENT, fe_kind=inputs.CAHN_HILLIARD, **kw):
    base = dict(nx=nx, ny=ny, nz=nz, h=1.0, flow_kind=flow_kind, u_max=0.0, v_lo=0.0,
                v_hi=0.0, eta=1.0, fe_kind=fe_kind, sigma=1.0, kappa=1.0, eps=1.0,
                mobility=1.0, k_area=0.0, k_vol=0.0)
    base.update(kw)
    return OracleParams(**base)


def _state(p, phi, psi=None, omega=None):
    """A state with the given fields and the wall data of p's body-free flow
    (no Poisson solve: the observables read the fields as given)."""
    bf = base_flow(p.flow_kind, p.nx, p.ny, p.nz, p.h, u_max=p.u_max, v_lo=p.v_lo,
                   v_hi=p.v_hi)
    shape = (p.nz, p.ny, p.nx)
    zero = [np.zeros(shape) for _ in range(3)]
    return OracleState(p=p, bf=bf, phi=np.array(phi, dtype=np.float64), mu=np.zeros(shape),
                       omega=omega if omega is not None else zero,
                       psi=psi if psi is not None else zero,
                       V0=0.0, A0=0.0, V=0.0, A=0.0, gamma_a=0.0)


# ------------------------------------------------------------ body-free channel flows
def test_couette_stress_dissipation_and_zero_resistance():
    """Body-free Couette (walls on the ghost nodes, H = (ny + 1) h): the
    discrete velocity is the linear profile, so every cell has shear rate
    g = (v_hi - v_lo) / H and no other gradient.  Then <sigma_xy>(y) = eta g
    in every row, sigma_t = |sigma_xy| everywhere, D = (eta/2) * 2 g^2 per
    unit volume summed over N cells = eta g^2 N h^3, D0 = D, resistance 0,
    no deviation from the body-free fields, and both divergences vanish."""
    nx, ny, nz, h = 6, 9, 4, 0.5
    vlo, vhi, eta = -0.05, 0.08, 0.3
    p = _params(nx, ny, nz, h=h, flow_kind=inputs.COUETTE, v_lo=vlo, v_hi=vhi, eta=eta)
    st = init_state(p, np.ones((nz, ny, nx)))
    d = diagnostics(st)
    g = (vhi - vlo) / ((ny + 1) * h)
    tau = eta * g
    assert np.max(np.abs(d["stress_profile"] - tau)) < 1e-14 * abs(tau) * 100
    assert np.max(np.abs(d["sigma_t"] - abs(tau))) < 1e-12 * abs(tau)
    assert abs(d["max_sigma_t"] - abs(tau)) < 1e-12 * abs(tau)
    D = eta * g * g * nx * ny * nz * h ** 3
    assert abs(d["dissipation"] / D - 1) < 1e-12
    assert abs(d["dissipation0"] / D - 1) < 1e-12
    assert abs(d["resistance_rel"]) < 1e-12
    assert d["omega_dev2"] < 1e-28 and d["psi_dev2"] < 1e-26
    assert d["max_div_v"] < 1e-15 and d["max_div_psi"] < 1e-15
    assert d["volume"] == 0.0 and d["area"] == 0.0


def test_planar_poiseuille_stress_profile_and_dissipation():
    """Planar Poiseuille, no body: the discrete velocity is
    v_x(y) = 4 U y (H - y) / H^2 - (4/3) U h^2 / H^2 (central difference of
    the cubic psi_z), so its central y-difference is the exact slope
    4 U (H - 2y) / H^2 in every row whose neighbours are cells.  In the two
    wall rows the no-slip wall value 0 replaces the profile's extension
    -(4/3) U h^2 / H^2, shifting the slope by -(2/3) U h / H^2 (row 0) and
    +(2/3) U h / H^2 (row ny - 1).  sigma_xy = eta * slope, and
    D = eta h^3 nx nz sum_j slope_j^2 (only d v_x / dy is non-zero)."""
    nx, ny, nz, h, U, eta = 4, 11, 3, 0.5, 0.07, 0.45
    p = _params(nx, ny, nz, h=h, flow_kind=inputs.POISEUILLE_PLANAR, u_max=U, eta=eta)
    st = init_state(p, np.ones((nz, ny, nx)))
    d = diagnostics(st)
    H = (ny + 1) * h
    y = (np.arange(ny) + 1.0) * h
    slope = 4 * U * (H - 2 * y) / H ** 2
    slope[0] -= 2.0 / 3.0 * U * h / H ** 2
    slope[-1] += 2.0 / 3.0 * U * h / H ** 2
    assert np.max(np.abs(d["stress_profile"] - eta * slope)) < 1e-15
    assert np.max(np.abs(d["sigma_t"] - np.abs(eta * slope)[None, :, None])) < 1e-15
    D = eta * h ** 3 * nx * nz * float(np.sum(slope ** 2))
    assert abs(d["dissipation"] / D - 1) < 1e-12
    assert abs(d["resistance_rel"]) < 1e-12
    assert d["max_div_v"] < 1e-15


# ------------------------------------------------------------ a trigonometric stream vector
class _Trig:
    """Sum of products c * f(a i) * f(b (j + 1)) * f(q k), f in {sin, cos};
    central differences act on it term by term through the sum-to-product
    identities of the module docstring."""

    def __init__(self, terms):
        self.terms = list(terms)   # (coef, (fx, a), (fy, b), (fz, q))

    def __add__(self, other):
        return _Trig(self.terms + other.terms)

    def __neg__(self):
        return _Trig([(-c, fx, fy, fz) for c, fx, fy, fz in self.terms])

    def d(self, axis, h):
        out = []
        for c, *fs in self.terms:
            kind, t = fs[axis]
            fs = list(fs)
            if kind == "s":
                fs[axis] = ("c", t)
                c2 = c * math.sin(t) / h
            else:
                fs[axis] = ("s", t)
                c2 = -c * math.sin(t) / h
            out.append((c2, *fs))
        return _Trig(out)

    def eval(self, nx, ny, nz):
        i = np.arange(nx)[None, None, :]
        j = (np.arange(ny) + 1.0)[None, :, None]
        k = np.arange(nz)[:, None, None]
        f = {"s": np.sin, "c": np.cos}
        out = np.zeros((nz, ny, nx))
        for c, (kx, a), (ky, b), (kz, q) in self.terms:
            out = out + c * f[kx](a * i) * f[ky](b * j) * f[kz](q * k)
        return out


def _wall_free_profile(fx, fz, b1, b2, coef):
    """c fx(.) fz(.) [sin(b1 (j+1)) / sin b1 - sin(b2 (j+1)) / sin b2]: zero on
    the wall nodes j = -1, n (b1, b2 multiples of pi / (n + 1)), and so is its
    central y-difference cos(b1 (j+1)) - cos(b2 (j+1)) when b1, b2 are odd
    (or even) multiples alike."""
    return _Trig([(coef / math.sin(b1), fx, ("s", b1), fz),
                  (-coef / math.sin(b2), fx, ("s", b2), fz)])


def _trig_flow(nx, ny, nz, h, wall_free):
    """Trigonometric stream vector and its velocity v = curl psi (eq. vecpot,
    central differences), both as _Trig sums.  psi vanishes on the wall
    nodes (its wall data are zero).  With wall_free the velocity vanishes
    there too; otherwise psi_x, psi_z are single sine modes in y and the
    velocity's closed form is non-zero on the wall nodes."""
    a, q = 2 * math.pi / nx, 2 * math.pi / nz
    b1, b2, b3 = math.pi / (ny + 1), 3 * math.pi / (ny + 1), 2 * math.pi / (ny + 1)
    if wall_free:
        px = _wall_free_profile(("c", a), ("c", q), b1, b2, 0.3)
        pz = _wall_free_profile(("s", 2 * a), ("s", q), b1, b2, 0.25)
    else:
        px = _Trig([(0.3, ("c", a), ("s", b1), ("c", q))])
        pz = _Trig([(0.25, ("s", 2 * a), ("s", b2), ("s", q))])
    py = _Trig([(-0.2, ("s", a), ("s", b3), ("c", q))])
    psi = (px, py, pz)
    vx = psi[2].d(1, h) + -psi[1].d(2, h)
    vy = psi[0].d(2, h) + -psi[2].d(0, h)
    vz = psi[1].d(0, h) + -psi[0].d(1, h)
    return psi, (vx, vy, vz)


def _eval_rows(t, nx, nz, rows):
    """Values of a _Trig sum on the y rows ``rows`` (j may be -1 or n)."""
    f = {"s": np.sin, "c": np.cos}
    i = np.arange(nx)[None, None, :]
    k = np.arange(nz)[:, None, None]
    j = np.asarray(rows, dtype=float)[None, :, None] + 1.0
    return sum(c * f[kx](a * i) * f[ky](b * j) * f[kz](qq * k)
               for c, (kx, a), (ky, b), (kz, qq) in t.terms)


@pytest.mark.parametrize("wall_free", [True, False])
def test_stress_tensor_and_dissipation_of_trig_flow(wall_free):
    """Walls at rest in y, x and z periodic, a trigonometric stream vector:
    every velocity derivative is a closed-form sum of trigonometric products.
    In the two wall rows the y-difference meets the no-slip wall velocity 0
    instead of the closed form's value v_w on the wall node, which adds
    +v_w(-1) / (2h) in row 0 and -v_w(n) / (2h) in row n - 1 (zero when the
    velocity vanishes on the wall nodes).  This fixes sigma_t (every
    component of the symmetric stress: a transposed or antisymmetric gradient
    fails), the dissipation, max |div psi| and the zero resistance of a flow
    at rest.  (Summation by parts gives sum G : G^T = sum (div_h v)^2 = 0 for
    any curl whose wall-normal velocity vanishes on the wall nodes, so D also
    equals eta h^3 sum |G|^2 here, as for incompressible no-slip flow.)"""
    nx, ny, nz, h, eta = 8, 7, 6, 0.7, 0.35
    p = _params(nx, ny, nz, h=h, flow_kind=inputs.COUETTE, eta=eta)   # v_lo = v_hi = 0
    psi_t, v_t = _trig_flow(nx, ny, nz, h, wall_free)
    psi = [f.eval(nx, ny, nz) for f in psi_t]
    d = diagnostics(_state(p, np.ones((nz, ny, nx)), psi=psi))
    G = [[v_t[i].d(j, h).eval(nx, ny, nz) for j in range(3)] for i in range(3)]
    for i in range(3):
        vw = _eval_rows(v_t[i], nx, nz, [-1, ny])
        if wall_free:
            assert np.max(np.abs(vw)) < 1e-15
        G[i][1][:, 0, :] += vw[:, 0, :] / (2 * h)
        G[i][1][:, -1, :] -= vw[:, 1, :] / (2 * h)
    sxy = eta * (G[0][1] + G[1][0])
    syz = eta * (G[1][2] + G[2][1])
    sxz = eta * (G[0][2] + G[2][0])
    st_ref = np.sqrt(sxy ** 2 + syz ** 2 + sxz ** 2)
    scale = float(np.max(st_ref))
    assert scale > 1e-3
    assert np.max(np.abs(d["sigma_t"] - st_ref)) < 1e-13 * scale
    assert abs(d["max_sigma_t"] - scale) < 1e-13 * scale
    assert np.max(np.abs(d["stress_profile"] - sxy.mean(axis=(0, 2)))) < 1e-14 * scale
    D = 0.5 * eta * h ** 3 * sum(float(np.sum((G[i][j] + G[j][i]) ** 2))
                                 for i in range(3) for j in range(3))
    assert abs(d["dissipation"] / D - 1) < 1e-12
    div_psi = (psi_t[0].d(0, h) + psi_t[1].d(1, h) + psi_t[2].d(2, h)).eval(nx, ny, nz)
    assert abs(d["max_div_psi"] - float(np.max(np.abs(div_psi)))) < 1e-14
    assert d["max_div_psi"] > 1e-2
    if wall_free:   # div curl = 0 identically, and the wall rows are exact
        assert d["max_div_v"] < 1e-14
    assert d["dissipation0"] == 0.0 and d["resistance_rel"] == 0.0


def test_flow_deviations_by_orthogonality():
    """int |psi - psi0|^2 and int |omega - omega0|^2 (results section) of
    trigonometric fields over a body-free flow at rest: sums of squared
    products of full-period harmonics are products of n/2 (periodic axis) and
    (n + 1)/2 (sine modes on a walled axis), so h^3 sum c^2 prod(...)."""
    nx, ny, nz, h = 8, 7, 6, 0.7
    p = _params(nx, ny, nz, h=h, flow_kind=inputs.COUETTE)
    a, q, b = 2 * math.pi / nx, 2 * math.pi / nz, 2 * math.pi / (ny + 1)
    fx = _Trig([(0.3, ("c", a), ("s", b), ("c", q))]).eval(nx, ny, nz)
    fz = _Trig([(0.25, ("s", 2 * a), ("s", b), ("s", q))]).eval(nx, ny, nz)
    om = _Trig([(0.5, ("c", 3 * a), ("s", 2 * b), ("c", q))]).eval(nx, ny, nz)
    zero = np.zeros((nz, ny, nx))
    st = _state(p, np.ones((nz, ny, nx)), psi=[fx, zero, fz], omega=[zero, om, zero])
    d = diagnostics(st)
    vol = (nx / 2) * ((ny + 1) / 2) * (nz / 2)
    assert abs(d["psi_dev2"] / (h ** 3 * (0.3 ** 2 + 0.25 ** 2) * vol) - 1) < 1e-13
    assert abs(d["omega_dev2"] / (h ** 3 * 0.5 ** 2 * vol) - 1) < 1e-13


# ------------------------------------------------------------ body observables
@pytest.mark.parametrize("flow_kind", [inputs.QUIESCENT, inputs.COUETTE])
def test_centre_of_mass_of_symmetric_body(flow_kind):
    """A sharp ball (phi = -1 within radius r of one cell's centre, +1
    elsewhere) is symmetric about that cell, so its centre of mass is the
    cell's coordinate: x = (i + 1/2) h on the periodic axis, (j + 1) h along
    a walled axis (walls on the ghost nodes), and z by the same rule for a
    walled or periodic z.  The volume is h^3 times the number of cells in it."""
    nx, ny, nz, h = 16, 12, 10, 0.5
    p = _params(nx, ny, nz, h=h, flow_kind=flow_kind)
    i0, j0, k0, r = 5, 4, 6, 2.2
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inside = (i - i0) ** 2 + (j - j0) ** 2 + (k - k0) ** 2 <= r * r
    phi = np.where(inside, -1.0, 1.0)
    d = diagnostics(_state(p, phi), with_reference=False)
    zper = flow_kind == inputs.COUETTE
    expect = ((i0 + 0.5) * h, (j0 + 1.0) * h, (k0 + (0.5 if zper else 1.0)) * h)
    assert np.max(np.abs(np.array(d["com"]) - np.array(expect))) < 1e-13
    assert abs(d["volume"] - h ** 3 * int(np.sum(inside))) < 1e-12


def _sphere_phi(n, h, R, eps):
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    m = n * h / 2
    r = np.sqrt((X - m) ** 2 + (Y - m) ** 2 + (Z - m) ** 2)
    return np.tanh((r - R) / (math.sqrt(2.0) * eps))


def test_reduced_volume_and_energies_of_sphere():
    """tanh sphere of radius R = 8 eps (SM eq. 10) at h = eps/2 and eps/4.

    Across the interface, (1 - phi)/2 is the step at r = R smoothed by the
    kernel sech^2(x/w) / (2w), w = sqrt(2) eps, of variance pi^2 w^2 / 12; the
    area density of SM eq. 32 on the equilibrium profile is the kernel
    (3 / (4 w)) sech^4(x/w) of unit mass and variance (pi^2 - 6) w^2 / 12.
    Integrating 4 pi r^2 against them: V = 4/3 pi (R^3 + 3 R pi^2 w^2 / 12),
    A = 4 pi (R^2 + (pi^2 - 6) w^2 / 12), so the reduced volume (SM eq. 40)
    of a finite-width sphere tends to V / (4/3 pi (A / 4 pi)^1.5) = 1.0610 at
    R = 8 eps (-> 1 as R / eps grows).  The Helfrich energy tends to
    8 pi kappa (eq. 30), a tension sigma adds sigma A, and the Cahn-Hilliard
    energy (sigma = eps^2) is gamma A with gamma = 2 sqrt(2 sigma) / 3
    (SM eq. 15).  The discrete values converge to these at second order;
    the bending energy's own limit differs from 8 pi kappa by O(eps^2/R^2)."""
    eps, R, kappa, tension = 1.0, 8.0, 1.3, 0.6
    w2 = 2 * eps * eps
    V = 4 / 3 * math.pi * (R ** 3 + 3 * R * math.pi ** 2 * w2 / 12)
    A = 4 * math.pi * (R * R + (math.pi ** 2 - 6) * w2 / 12)
    vr_lim = V / (4 / 3 * math.pi * (A / (4 * math.pi)) ** 1.5)
    gamma = 2 * math.sqrt(2.0) / 3
    errs = []
    for h in (0.5, 0.25):
        n = int(round(2 * (R + 6 * eps) / h))
        phi = _sphere_phi(n, h, R, eps)
        p = _params(n, n, n, h=h, fe_kind=inputs.HELFRICH, kappa=kappa, eps=eps, sigma=0.0)
        d = diagnostics(_state(p, phi), with_reference=False)
        p.sigma = tension
        dt = diagnostics(_state(p, phi), with_reference=False)
        pc = _params(n, n, n, h=h, fe_kind=inputs.CAHN_HILLIARD, sigma=eps * eps, eps=eps)
        dc = diagnostics(_state(pc, phi), with_reference=False)
        assert abs(d["volume"] / V - 1) < 1e-4
        errs.append([abs(d["area"] / A - 1), abs(d["reduced_volume"] - vr_lim),
                     abs(d["energy"] / (8 * math.pi * kappa) - 1),
                     abs((dt["energy"] - d["energy"]) / (tension * A) - 1),
                     abs(dc["energy"] / (gamma * A) - 1)])
    assert max(errs[0]) < 0.02 and max(errs[1]) < 0.005, errs
    # area, V_r, tension and CH energies: second-order discretisation error
    for e0, e1 in zip(errs[0][:2] + errs[0][3:], errs[1][:2] + errs[1][3:]):
        assert 1.7 < math.log2(e0 / e1) < 2.3, errs
    # the bending energy of a finite-width sphere also differs from 8 pi
    # kappa by O(eps^2 / R^2): within 1 % and closer on the finer grid
    assert errs[0][2] < 0.01 and errs[1][2] < errs[0][2], errs
