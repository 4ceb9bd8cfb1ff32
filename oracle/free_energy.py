"""Chemical potential, energies and the volume / area functionals (oracle).

* Cahn-Hilliard (eq. 31, SM eq. 1c): F = int 1/4 (phi^2 - 1)^2 +
  sigma/2 |grad phi|^2,  mu = phi^3 - phi - sigma lap phi.
* Phase-field Helfrich with C0 = 0 (eq. 30): F = C_F int g^2 with
  g = phi^3 - phi - eps^2 lap phi and C_F = 3 sqrt(2) kappa / (8 eps^3).
  Its functional derivative by the rule of SM eq. 34 is
  mu = 2 C_F [(3 phi^2 - 1) g - eps^2 lap g]; the supplementary material
  prints this with the prefactor 3 sqrt(2) kappa / (4 eps^3) (= 2 C_F) in
  the Helfrich-case paragraph and with 3 sqrt(2) kappa / (8 eps^3) in
  SM eq. 35.  The oracle takes the exact derivative (2 C_F); a flag selects
  the SM eq. 35 reading.  The area term of SM eq. 35, -gamma_A lap phi, is
  added as printed, with the penalty multiplier
  gamma_A = K_A (A - A0) * 3 eps / (2 sqrt 2) (the coefficient of lap phi in
  the derivative of the area functional SM eq. 32).
* Membrane tension (Helfrich kind with sigma != 0): F = C_F int g^2 +
  sigma A_f[phi], where A_f is the area functional of SM eq. 32 with the
  gradient summed over cell faces; its derivative adds (c_A / eps) sigma g to
  mu.  Reading: the paper treats tension (Cahn-Hilliard) and bending
  (Helfrich) as alternatives; the combination is the tension-plus-bending
  energy of a membrane, F_m(kappa) + sigma A, with sigma the tension.
* Area functional (SM eq. 32): A = 3/(2 sqrt 2) int eps/2 |grad phi|^2 +
  (phi^2 - 1)^2 / (4 eps), with central differences for grad phi.
* Volume (SM eq. 37 with phi = -1 inside the body): V = 1/2 int (1 - phi).

Discrete definitions use the face-mirror (no-flux) ghosts of ``grid``.

Pinned by: exact discrete energy-gradient identity mu_i = h^-3 dF_h/dphi_i
(central finite differences of F_h), flat tanh interface, tanh sphere area
-> 4 pi R^2 and Helfrich energy -> 8 pi kappa, Gibbs-Thomson mu = gamma H,
mu of the tension-plus-bending energy = h^-3 d(F_h + sigma A_f)/dphi_i.
"""
from __future__ import annotations

import math

import numpy as np

from inputs import CAHN_HILLIARD, HELFRICH
from .grid import pad_mirror, lap, grad


def prefactor_cf(kappa: float, eps: float) -> float:
    """C_F = 3 sqrt(2) kappa / (8 eps^3) of eq. 30."""
    return 3.0 * math.sqrt(2.0) * kappa / (8.0 * eps ** 3)


def helfrich_g(phi, eps, h, zper):
    return phi ** 3 - phi - eps * eps * lap(pad_mirror(phi, 1, zper), h)


def chem_potential(phi, fe_kind, h, zper, sigma=0.0, kappa=0.0, eps=1.0, gamma_a=0.0,
                   mu_prefactor_half=False):
    if fe_kind == CAHN_HILLIARD:
        return phi ** 3 - phi - sigma * lap(pad_mirror(phi, 1, zper), h)
    if fe_kind != HELFRICH:
        raise ValueError("unknown free-energy kind")
    g = helfrich_g(phi, eps, h, zper)
    lap_g = lap(pad_mirror(g, 1, zper), h)
    pref = prefactor_cf(kappa, eps) * (1.0 if mu_prefactor_half else 2.0)
    mu = pref * ((3.0 * phi ** 2 - 1.0) * g - eps * eps * lap_g)
    if gamma_a != 0.0:
        mu = mu - gamma_a * lap(pad_mirror(phi, 1, zper), h)
    if sigma != 0.0:
        mu = mu + sigma * tension_mu_coefficient(eps) * g
    return mu


def tension_mu_coefficient(eps):
    """c_A / eps with c_A = 3 / (2 sqrt 2): the membrane tension sigma adds
    sigma * A_f[phi] to the Helfrich energy, and the derivative of the
    face-difference area A_f (``area_faces``) is (c_A / eps) g."""
    return 3.0 / (2.0 * math.sqrt(2.0) * eps)


def area_faces(phi, eps, h, zper):
    """Area functional of SM eq. 32 with |grad phi|^2 summed over cell faces
    (forward differences, as in ``ch_energy``): A_f = (c_A / eps) *
    h^3 sum [1/4 (phi^2 - 1)^2 + eps^2 / 2 sum_faces (D+ phi)^2], i.e. the
    Cahn-Hilliard energy with gradient coefficient eps^2 scaled by c_A / eps.
    Its exact discrete gradient h^-3 dA_f/dphi = (c_A / eps) (phi^3 - phi -
    eps^2 lap phi) = (c_A / eps) g."""
    return tension_mu_coefficient(eps) * ch_energy(phi, eps * eps, h, zper)


def volume(phi, h):
    """Body volume V = (h^3 / 2) sum (1 - phi)."""
    return 0.5 * h ** 3 * float(np.sum(1.0 - phi))


def area_density(phi, eps, h, zper):
    gx, gy, gz = grad(pad_mirror(phi, 1, zper), h)
    return (3.0 / (2.0 * math.sqrt(2.0))) * (
        0.5 * eps * (gx * gx + gy * gy + gz * gz) + (phi * phi - 1.0) ** 2 / (4.0 * eps))


def area(phi, eps, h, zper):
    return h ** 3 * float(np.sum(area_density(phi, eps, h, zper)))


def area_multiplier(k_area, a, a0, eps):
    """gamma_A = K_A (A - A0) * 3 eps / (2 sqrt 2)."""
    return k_area * (a - a0) * 3.0 * eps / (2.0 * math.sqrt(2.0))


def volume_multiplier(k_vol, v, v0):
    """lambda_V = K_V (V - V0): positive when the body is too large, which
    raises phi everywhere and shrinks the phi < 0 region."""
    return k_vol * (v - v0)


def helfrich_energy(phi, kappa, eps, h, zper):
    """F_h = C_F h^3 sum g^2 (eq. 30 without the area term)."""
    g = helfrich_g(phi, eps, h, zper)
    return prefactor_cf(kappa, eps) * h ** 3 * float(np.sum(g * g))


def ch_energy(phi, sigma, h, zper):
    """F_h = h^3 sum [1/4 (phi^2-1)^2 + sigma/2 sum_faces (D+ phi)^2]; the
    forward differences run over every face whose both cells exist (mirror
    faces carry zero gradient, periodic faces wrap)."""
    nz, ny, nx = phi.shape
    bulk = 0.25 * (phi * phi - 1.0) ** 2
    dx = (np.roll(phi, -1, axis=2) - phi) / h       # x periodic: all nx faces
    dy = (phi[:, 1:, :] - phi[:, :-1, :]) / h
    if zper:
        dz = (np.roll(phi, -1, axis=0) - phi) / h
    else:
        dz = (phi[1:, :, :] - phi[:-1, :, :]) / h
    grad2 = float(np.sum(dx * dx)) + float(np.sum(dy * dy)) + float(np.sum(dz * dz))
    return h ** 3 * (float(np.sum(bulk)) + 0.5 * sigma * grad2)
