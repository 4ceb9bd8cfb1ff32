"""Seeded synthetic workloads for the vorticity--stream-vector phase-field step.

This module is shared by the CPU oracle and the GPU path, and therefore holds
none of the method's arithmetic: no Laplacian, no chemical potential, no
Poisson solve, no base flow.  It only produces

* grid shapes and physical parameters for named workloads, and
* the initial order parameter phi0 = tanh(d / (sqrt(2) eps)) of a sphere or a
  prolate ellipsoid (d = approximate signed distance, positive outside, so
  that phi = -1 inside the body as in the matched-asymptotics section of the
  supplementary material, eqs. SM 9-10).

Coordinates (shared convention, stated once here so both sides agree):
arrays are C-ordered ``[nz][ny][nx]``; x is the periodic flow axis.  Along a
walled axis the flow walls sit on the ghost nodes j = -1 and j = n, so cell j
has coordinate (j + 1) h and the channel height is (n + 1) h.  Along a periodic
axis cell i has coordinate (i + 1/2) h.

Parameter derivations that are not the method (capillary number -> viscosity,
reduced volume -> ellipsoid axes) use closed-form continuum formulas:
surface tension gamma = 2 sqrt(2 sigma) / 3 (SM eq. 15), bending time
tau_kappa = eta V / kappa (main text eq. tau_k), reduced volume (SM eq. 40)
with the closed-form prolate-spheroid volume and area.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np

# flow kinds (same integer values as the C enum vsv_flow_kind)
POISEUILLE_DUCT = 0
POISEUILLE_PLANAR = 1
COUETTE = 2
QUIESCENT = 3

# free-energy kinds (C enum vsv_fe_kind)
CAHN_HILLIARD = 0
HELFRICH = 1


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    flow_kind: int
    u_max: float          # Poiseuille centre-line speed target
    v_lo: float           # Couette wall speed at the y = 0 wall (along x)
    v_hi: float           # Couette wall speed at the y = H wall (along x)
    eta: float
    fe_kind: int
    sigma: float          # Cahn-Hilliard gradient coefficient
    kappa: float          # bending modulus
    eps: float            # interface width parameter
    mobility: float
    k_area: float         # area penalty stiffness K_A
    k_vol: float          # volume penalty stiffness K_V
    dt: float
    nsteps: int
    seed: int
    body: dict = field(default_factory=dict)   # geometry actually drawn
    phi0: Optional[np.ndarray] = None          # float64 [nz][ny][nx]
    rho: float = 0.0                           # fluid density (0: no inertia)
    # time-dependent walls: (ramp, amplitude, frequency, phase), each a pair
    # (wall 0, wall 1), or None for steady walls
    wall_motion: Optional[tuple] = None

    @property
    def z_periodic(self) -> bool:
        return self.flow_kind in (COUETTE, POISEUILLE_PLANAR)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def params(self) -> dict:
        d = asdict(self)
        d.pop("phi0")
        return d


# ---------------------------------------------------------------- geometry
def cell_coords(n: int, h: float, walled: bool) -> np.ndarray:
    """Cell-centre coordinates along one axis (see module docstring)."""
    j = np.arange(n, dtype=np.float64)
    return (j + 1.0) * h if walled else (j + 0.5) * h


def channel_extent(n: int, h: float, walled: bool) -> float:
    return (n + 1) * h if walled else n * h


def prolate_volume(a: float, b: float) -> float:
    return 4.0 / 3.0 * math.pi * a * b * b


def prolate_area(a: float, b: float) -> float:
    if a <= b:
        return 4.0 * math.pi * b * b
    e = math.sqrt(1.0 - (b * b) / (a * a))
    return 2.0 * math.pi * b * b * (1.0 + a / (b * e) * math.asin(e))


def reduced_volume(a: float, b: float) -> float:
    """SM eq. 40 with the closed-form spheroid volume and area."""
    V = prolate_volume(a, b)
    A = prolate_area(a, b)
    return V / (4.0 / 3.0 * math.pi * (A / (4.0 * math.pi)) ** 1.5)


def prolate_axis_for(vr: float, b: float) -> float:
    """Long semi-axis a >= b with reduced_volume(a, b) == vr (bisection)."""
    lo, hi = b, 50.0 * b
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if reduced_volume(mid, b) > vr:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def ellipsoid_phi(nx, ny, nz, h, z_periodic, centre, axes, eps) -> np.ndarray:
    """phi0 = tanh(d / (sqrt(2) eps)); d ~ (rho - 1) / |grad rho|,
    rho^2 = sum (x_i / a_i)^2 (exact signed distance for a sphere)."""
    x = cell_coords(nx, h, False)
    y = cell_coords(ny, h, True)
    z = cell_coords(nz, h, not z_periodic)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ax, ay, az = axes
    qx, qy, qz = (X - centre[0]) / ax, (Y - centre[1]) / ay, (Z - centre[2]) / az
    rho = np.sqrt(qx * qx + qy * qy + qz * qz)
    rho_safe = np.maximum(rho, 1e-300)
    grad = np.sqrt((qx / ax) ** 2 + (qy / ay) ** 2 + (qz / az) ** 2) / rho_safe
    d = np.where(rho > 0, (rho - 1.0) / np.maximum(grad, 1e-300), -min(axes))
    return np.tanh(d / (math.sqrt(2.0) * eps))


def channel_centre(nx, ny, nz, h, z_periodic):
    return (channel_extent(nx, h, False) / 2.0,
            channel_extent(ny, h, True) / 2.0,
            channel_extent(nz, h, not z_periodic) / 2.0)


def surface_tension(sigma: float) -> float:
    """gamma = 2 sqrt(2 sigma) / 3 (SM eq. 15)."""
    return 2.0 * math.sqrt(2.0 * sigma) / 3.0


def stable_k_vol(dt, mobility, ncells, h, factor=0.5):
    """Volume-penalty stiffness whose explicit relaxation factor per step,
    dt * M * K_V * N * h^3 / 2, equals ``factor`` (must stay below 2)."""
    return 2.0 * factor / (dt * mobility * ncells * h ** 3)


# ---------------------------------------------------------------- workloads
def droplet_duct(nx=48, ny=24, nz=24, radius=6.0, seed=0, nsteps=10, dt=0.01,
                 u_max=0.05, ca=0.1, sigma=1.0, eps=1.0, flow_kind=POISEUILLE_DUCT,
                 name="droplet_duct") -> Workload:
    """Cahn-Hilliard droplet of given radius at the channel centre, duct
    Poiseuille flow; eta from Ca = eta U / gamma.  Deterministic (seed only
    recorded)."""
    h = 1.0
    gamma = surface_tension(sigma)
    eta = ca * gamma / u_max if u_max > 0 else 1.0
    zper = flow_kind in (COUETTE, POISEUILLE_PLANAR)
    c = channel_centre(nx, ny, nz, h, zper)
    phi0 = ellipsoid_phi(nx, ny, nz, h, zper, c, (radius,) * 3, eps)
    return Workload(name=name, nx=nx, ny=ny, nz=nz, h=h, flow_kind=flow_kind,
                    u_max=u_max, v_lo=0.0, v_hi=0.0, eta=eta, fe_kind=CAHN_HILLIARD,
                    sigma=sigma, kappa=0.0, eps=eps, mobility=1.0, k_area=0.0,
                    k_vol=0.0, dt=dt, nsteps=nsteps, seed=seed,
                    body={"centre": c, "axes": (radius,) * 3}, phi0=phi0)


def vesicle(nx, ny, nz, flow_kind, vr, eps, seed=0, nsteps=10, dt=1e-4,
            u_max=0.05, v_wall=0.05, ca=1.0, kappa=1.0, k_area=0.05,
            vol_factor=0.5, b_range=(0.11, 0.16), name="vesicle", b_ref=None) -> Workload:
    """Prolate Helfrich vesicle with seeded equatorial semi-axis b ~
    U(b_range) * b_ref (default ny) and long axis a (along x) fixed by the
    reduced volume.  eta from Ca = tau_kappa * shear_rate, tau_kappa = eta V /
    kappa."""
    h = 1.0
    rng = np.random.default_rng(seed)
    b = float(rng.uniform(*b_range)) * (ny if b_ref is None else b_ref) * h
    a = prolate_axis_for(vr, b)
    zper = flow_kind in (COUETTE, POISEUILLE_PLANAR)
    c = channel_centre(nx, ny, nz, h, zper)
    phi0 = ellipsoid_phi(nx, ny, nz, h, zper, c, (a, b, b), eps)
    H = channel_extent(ny, h, True)
    if flow_kind == COUETTE:
        shear = 2.0 * v_wall / H
        v_lo, v_hi, umax = -v_wall, v_wall, 0.0
    elif flow_kind in (POISEUILLE_DUCT, POISEUILLE_PLANAR):
        shear = 4.0 * u_max / H
        v_lo = v_hi = 0.0
        umax = u_max
    else:
        shear, v_lo, v_hi, umax = 0.0, 0.0, 0.0, 0.0
    vol = prolate_volume(a, b)
    eta = ca * kappa / (vol * shear) if shear > 0 else 1.0
    ncells = nx * ny * nz
    return Workload(name=name, nx=nx, ny=ny, nz=nz, h=h, flow_kind=flow_kind,
                    u_max=umax, v_lo=v_lo, v_hi=v_hi, eta=eta, fe_kind=HELFRICH,
                    sigma=0.0, kappa=kappa, eps=eps, mobility=1.0, k_area=k_area,
                    k_vol=stable_k_vol(dt, 1.0, ncells, h, vol_factor), dt=dt,
                    nsteps=nsteps, seed=seed,
                    body={"centre": c, "axes": (a, b, b), "reduced_volume": vr},
                    phi0=phi0)


def droplet_24x24x48(seed=0) -> Workload:
    """Plain FP64 droplet workload: 48x24x24 (x flow axis), duct Poiseuille
    U = 0.05, CH sigma = 1, eps = 1, Ca = 0.1, R = 6, 10 steps of dt = 0.01."""
    return droplet_duct(seed=seed, name="droplet_duct_48x24x24")


def vesicle_poiseuille_256x128x128(seed=0, nx=256, ny=128, nz=128, nsteps=2000) -> Workload:
    """Helfrich vesicle, V_r = 0.8, eps = 1, duct Poiseuille at Ca = 1."""
    return vesicle(nx, ny, nz, POISEUILLE_DUCT, 0.8, 1.0, seed=seed, nsteps=nsteps,
                   name=f"vesicle_duct_{nx}x{ny}x{nz}")


def vesicle_poiseuille_128x64x64(seed=0, nx=128, ny=64, nz=64, nsteps=200) -> Workload:
    """Differentiable run: Helfrich vesicle, V_r = 0.8, eps = 1, duct
    Poiseuille at Ca = 1, kappa = 1 and no tension as the starting point of a
    parameter fit."""
    return vesicle(nx, ny, nz, POISEUILLE_DUCT, 0.8, 1.0, seed=seed, nsteps=nsteps,
                   name=f"vesicle_duct_{nx}x{ny}x{nz}")


def vesicle_couette_512x256x256(seed=0, nx=512, ny=256, nz=256, nsteps=500) -> Workload:
    """Helfrich vesicle, V_r = 0.9, eps = 1.5, Couette walls at +-0.05."""
    return vesicle(nx, ny, nz, COUETTE, 0.9, 1.5, seed=seed, nsteps=nsteps,
                   name=f"vesicle_couette_{nx}x{ny}x{nz}")


def batch_instances(n=64, seed=0, dt=1e-4, nsteps=60) -> list:
    """Independent problems of a parameter sweep (batched stepping): sizes
    multiples of 8 with ny, nz in [32, 96] and nx in [32, 192]; Ca log-uniform
    in [0.05, 5]; half spherical Cahn-Hilliard droplets (radius a quarter of
    the smallest extent), half Helfrich vesicles with V_r ~ U(0.7, 0.98) and
    the body sized by the smallest extent (nx / 3 for the long axis); duct
    Poiseuille or Couette flow, 50/50.  All with eps = 1 and step dt."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ny = 8 * int(rng.integers(4, 13))
        nz = 8 * int(rng.integers(4, 13))
        nx = 8 * int(rng.integers(4, 25))
        ca = float(math.exp(rng.uniform(math.log(0.05), math.log(5.0))))
        flow = POISEUILLE_DUCT if rng.uniform() < 0.5 else COUETTE
        if rng.uniform() < 0.5:
            r = 0.25 * min(nx, ny, nz)
            w = droplet_duct(nx=nx, ny=ny, nz=nz, radius=r, seed=seed, nsteps=nsteps, dt=dt,
                             ca=ca, flow_kind=flow, name=f"batch{i}_droplet_{nx}x{ny}x{nz}")
            if flow == COUETTE:   # Ca = eta gamma_dot R / gamma with the wall shear rate
                shear = 2.0 * 0.05 / channel_extent(ny, 1.0, True)
                w.u_max, w.v_lo, w.v_hi = 0.0, -0.05, 0.05
                w.eta = ca * surface_tension(w.sigma) / (shear * r)
        else:
            vr = float(rng.uniform(0.7, 0.98))
            ref = min(ny, nz, nx / 3.0)
            w = vesicle(nx, ny, nz, flow, vr, 1.0, seed=seed + i, nsteps=nsteps, dt=dt, ca=ca,
                        b_range=(0.2, 0.3), b_ref=ref, name=f"batch{i}_vesicle_{nx}x{ny}x{nz}")
        out.append(w)
    return out


def random_field(shape, seed, scale=1.0) -> np.ndarray:
    """Seeded standard-normal float64 field (for solver and operator tests)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
