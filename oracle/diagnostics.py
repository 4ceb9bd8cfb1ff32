"""Observables of the flow and the body (oracle, FP64).

* In-plane stress (in-plane-shear section): sigma_ij = eta (d_j v_i + d_i v_j),
  sigma_t = sqrt(sigma_xy^2 + sigma_yz^2 + sigma_xz^2); the stress profile is
  <sigma_xy> averaged over x and z as a function of y.
* Dissipation D = (eta / 2) int sum_ij (d_j v_i + d_i v_j)^2 dV and the
  relative hydrodynamic resistance (D - D0) / D0 against the body-free flow
  (the paper names the resistance but gives no formula; this is the reading
  for velocity-driven walls).
* Flow observables of the results section: int |omega - omega0|^2 dV and
  int |psi - psi0|^2 dV (the paper's xi is psi), omega0 / psi0 being the
  body-free fields.
* V, A, reduced volume V_r = V / (4/3 pi (A / 4 pi)^{3/2}) (SM eq. 40),
  bending (or Cahn-Hilliard) energy, centre of mass of the body
  (weights (1 - phi)/2), max |div v| and max |div psi|.

Velocity derivatives use central differences with the no-slip wall velocity
on the wall nodes.

Pinned by (tests/test_oracle_diagnostics_pins.py): the body-free Couette flow
(uniform <sigma_xy> = eta (v_hi - v_lo) / H, sigma_t = |sigma_xy|,
D = D0 = eta g^2 N h^3, zero resistance and deviations); the body-free planar
Poiseuille profile (linear <sigma_xy>(y) with its wall-row offsets, D from
it); a trigonometric stream vector whose stress tensor, dissipation and
max |div psi| are closed forms of the discrete calculus (with and without
velocity on the wall nodes); flow deviations of trigonometric fields by
orthogonality; the centre of mass of a sharp ball on any cell; the tanh
sphere's volume, area, reduced volume and energies against their
finite-width closed forms at second order.
"""
from __future__ import annotations

import math

import numpy as np

from inputs import CAHN_HILLIARD, cell_coords
from .grid import pad_flow, grad
from .flow import body_free_fields
from .free_energy import volume, area, helfrich_energy, ch_energy, area_faces
from .step import velocity


def velocity_gradient(v, vel_b, h, zper):
    """G[i][j] = d v_i / d x_j."""
    return [list(grad(pad_flow(v[i], vel_b[i], zper), h)) for i in range(3)]


def dissipation_of(v, vel_b, h, eta, zper):
    G = velocity_gradient(v, vel_b, h, zper)
    s = 0.0
    for i in range(3):
        for j in range(3):
            e = G[i][j] + G[j][i]
            s += float(np.sum(e * e))
    return 0.5 * eta * h ** 3 * s


def diagnostics(st, with_reference=True):
    p = st.p
    h, zp = p.h, p.z_periodic
    v = velocity(st)
    G = velocity_gradient(v, st.bf.vel_b, h, zp)
    sxy = p.eta * (G[0][1] + G[1][0])
    syz = p.eta * (G[1][2] + G[2][1])
    sxz = p.eta * (G[0][2] + G[2][0])
    sigma_t = np.sqrt(sxy * sxy + syz * syz + sxz * sxz)
    D = 0.0
    for i in range(3):
        for j in range(3):
            e = G[i][j] + G[j][i]
            D += float(np.sum(e * e))
    D *= 0.5 * p.eta * h ** 3
    V = volume(st.phi, h)
    A = area(st.phi, p.eps, h, zp)
    vr = V / (4.0 / 3.0 * math.pi * (A / (4.0 * math.pi)) ** 1.5) if A > 0 else 0.0
    if p.fe_kind == CAHN_HILLIARD:
        energy = ch_energy(st.phi, p.sigma, h, zp)
    else:
        energy = helfrich_energy(st.phi, p.kappa, p.eps, h, zp)
        if p.sigma != 0.0:   # membrane tension times the face-difference area
            energy += p.sigma * area_faces(st.phi, p.eps, h, zp)
    w = 0.5 * (1.0 - st.phi)
    wsum = float(np.sum(w))
    xs = cell_coords(p.nx, h, False)
    ys = cell_coords(p.ny, h, True)
    zs = cell_coords(p.nz, h, not zp)
    com = (float(np.sum(w * xs[None, None, :])) / wsum if wsum else 0.0,
           float(np.sum(w * ys[None, :, None])) / wsum if wsum else 0.0,
           float(np.sum(w * zs[:, None, None])) / wsum if wsum else 0.0)
    div_v = G[0][0] + G[1][1] + G[2][2]
    gpsi = [grad(pad_flow(st.psi[c], st.bf.psi_b[c], zp), h) for c in range(3)]
    div_psi = gpsi[0][0] + gpsi[1][1] + gpsi[2][2]
    out = {
        "volume": V, "area": A, "reduced_volume": vr, "energy": energy,
        "com": com, "dissipation": D,
        "max_div_v": float(np.max(np.abs(div_v))),
        "max_div_psi": float(np.max(np.abs(div_psi))),
        "max_sigma_t": float(np.max(sigma_t)),
        "stress_profile": sxy.mean(axis=(0, 2)),
        "sigma_t": sigma_t,
    }
    if with_reference:
        om0, ps0 = body_free_fields(st.bf, p.nx, p.ny, p.nz, h)
        out["omega_dev2"] = h ** 3 * sum(float(np.sum((st.omega[c] - om0[c]) ** 2)) for c in range(3))
        out["psi_dev2"] = h ** 3 * sum(float(np.sum((st.psi[c] - ps0[c]) ** 2)) for c in range(3))
        from .grid import curl
        v0 = curl(ps0, st.bf.psi_b, h, zp)
        D0 = dissipation_of(v0, st.bf.vel_b, h, p.eta, zp)
        out["dissipation0"] = D0
        out["resistance_rel"] = (D - D0) / D0 if D0 > 0 else 0.0
    return out
