"""Discrete adjoint of the forward step (oracle, FP64).

TEST INFRASTRUCTURE ONLY, like the rest of this package.

What it differentiates: the map (phi^0, kappa, sigma) -> phi^N of N steps
of ``step.step`` started by ``step.init_state`` (which fixes V0 = V[phi^0],
A0 = A[phi^0], mu^0 = mu(phi^0) and psi^0 from phi^0), and the shape loss

    J = h^3 / 2 * sum (phi^N - phi_target)^2.

Reverse mode of the discrete equations (differentiate the discrete step, not
the continuum equations), so the gradient is the derivative of the oracle's
own forward map up to rounding.  Step n -> n+1 in the order of ``step.step``:

    lambda^n   = K_V (V[phi^n] - V0)
    phi^{n+1}  = phi^n + dt [M (L_m mu^n + lambda^n) - v^n . D_m phi^n]
    gamma^{n+1}= K_A c_g (A[phi^{n+1}] - A0),           c_g = 3 eps / (2 sqrt 2)
    mu^{n+1}   = mu(phi^{n+1}; gamma^{n+1}, kappa, sigma)
    f          = (D_m phi^{n+1} x D_m mu^{n+1}) / eta
    omega      = omega_lift + L^-1 f,   psi^{n+1} = psi_lift + L^-1 (-omega)
    v^{n+1}    = curl psi^{n+1}

(L_m: 7-point Laplacian with mirror ghosts; D_m: central differences with
mirror ghosts; L: 7-point Laplacian with zero data on the walls; the lifts
carry the constant wall data.)  Transposes, all with respect to the plain
sum over cells:

* L_m and L are symmetric, so the adjoint Poisson problem is the same
  problem (the adjoint of psi -> omega -> f is two solves with L);
* D_m^T w = -D_odd w, the central difference of w with odd ghosts
  (w_{-1} = -w_0 at a mirror face, wrap on periodic axes);
* curl with zero ghosts on the walls is symmetric: curl^T = curl;
* d mu / d phi is symmetric: Helfrich cf2 [diag(6 phi g) + G G] + beta G -
  gamma L_m with G = diag(3 phi^2 - 1) - eps^2 L_m, beta = sigma c_A / eps;
  Cahn-Hilliard diag(3 phi^2 - 1) - sigma L_m;
* dV/dphi_i = -h^3 / 2; dA/dphi = h^3 c_A [eps D_m^T D_m phi +
  (phi^2 - 1) phi / eps], c_A = 3 / (2 sqrt 2).

The initial state has gamma^0 = 0 identically (A[phi^0] - A0 = 0 for every
phi^0), so only mu^0's explicit phi dependence and the flow solve enter
there, and the constants V0, A0 pass their adjoints back to phi^0.

Inertial variant (rho > 0): omega^{n+1} = omega_lift + (L - s)^-1 (f -
s omega^n), s = rho / (eta dt), so the adjoint of omega is carried from step
to step: fbar = (L - s)^-1 omegabar_total and omegabar^n = -s fbar.  The
initial vorticity is the Stokes one (L^-1 f^0).

Pinned by (tests/test_oracle_pins.py): dot-product identities of each
transpose against the forward operator it transposes; the vector-Jacobian
product of mu against central differences of ``chem_potential``; the
trajectory gradient in kappa, sigma and random directions of phi^0 against
central differences of the forward oracle (Helfrich with tension, the
area and volume penalties, duct and Couette flows, the inertial variant,
and Cahn-Hilliard).
"""
from __future__ import annotations

import math

import numpy as np

from inputs import CAHN_HILLIARD, HELFRICH
from .grid import pad_mirror, pad_homogeneous, lap, grad
from .poisson import solve_poisson
from .free_energy import prefactor_cf, helfrich_g
from .step import init_state, step, velocity, inertial_shift

C_A = 3.0 / (2.0 * math.sqrt(2.0))


# ---------------------------------------------------------------- transposes
def pad_odd(u: np.ndarray, z_periodic: bool) -> np.ndarray:
    """One ghost layer: x periodic, y (and z unless periodic) odd mirror
    about the wall face, ghost -1 <-> -u[0], ghost n <-> -u[n-1]."""
    P = pad_mirror(u, 1, z_periodic)
    P[:, 0, :] *= -1.0
    P[:, -1, :] *= -1.0
    if not z_periodic:
        P[0, :, :] *= -1.0
        P[-1, :, :] *= -1.0
    return P


def grad_mirror_t(w, h: float, z_periodic: bool) -> np.ndarray:
    """sum_a D_a^T w_a for the mirror central differences D_a of
    ``grid.grad(pad_mirror(.))``: minus the odd-ghost divergence."""
    out = -grad(pad_odd(w[0], z_periodic), h)[0]
    out -= grad(pad_odd(w[1], z_periodic), h)[1]
    out -= grad(pad_odd(w[2], z_periodic), h)[2]
    return out


def curl_zero(w, h: float, z_periodic: bool):
    """curl with zero ghosts on the walled axes (the homogeneous part of the
    velocity of a stream vector); it is its own transpose."""
    per = (True, False, z_periodic)
    g = [grad(pad_homogeneous(w[c], per), h) for c in range(3)]
    return [g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]]


def lap_m(u, h, z_periodic):
    return lap(pad_mirror(u, 1, z_periodic), h)


def cf2_of(p) -> float:
    """Prefactor of the bending mu: 2 C_F (C_F with the SM eq. 35 reading)."""
    cf = prefactor_cf(p.kappa, p.eps)
    return cf if p.mu_prefactor_half else 2.0 * cf


def area_grad(phi, p) -> np.ndarray:
    """dA/dphi of the central-difference area of SM eq. 32."""
    zp = p.z_periodic
    d = grad(pad_mirror(phi, 1, zp), p.h)
    return p.h ** 3 * C_A * (p.eps * grad_mirror_t(d, p.h, zp) + (phi * phi - 1.0) * phi / p.eps)


# ---------------------------------------------------------------- vector-Jacobian products
def mu_vjp(phi, gamma_a, mubar, p):
    """Adjoint of mu = mu(phi; gamma_A, kappa, sigma) for the adjoint mubar.

    Returns (phibar, kappabar, sigmabar, gammabar): (d mu / d phi)^T mubar
    and the sums <d mu / d kappa, mubar>, <d mu / d sigma, mubar>,
    <d mu / d gamma_A, mubar> over the cells."""
    h, zp = p.h, p.z_periodic
    lphi = lap_m(phi, h, zp)
    if p.fe_kind == CAHN_HILLIARD:
        phibar = (3.0 * phi * phi - 1.0) * mubar - p.sigma * lap_m(mubar, h, zp)
        return phibar, 0.0, float(np.sum(-lphi * mubar)), 0.0
    if p.fe_kind != HELFRICH:
        raise ValueError("unknown free-energy kind")
    e2 = p.eps * p.eps
    g = helfrich_g(phi, p.eps, h, zp)
    cf2 = cf2_of(p)
    beta = p.sigma * C_A / p.eps
    w = (3.0 * phi * phi - 1.0) * mubar - e2 * lap_m(mubar, h, zp)          # G mubar
    gw = (3.0 * phi * phi - 1.0) * w - e2 * lap_m(w, h, zp)                  # G G mubar
    phibar = cf2 * (6.0 * phi * g * mubar + gw) + beta * w - gamma_a * lap_m(mubar, h, zp)
    inner = (3.0 * phi * phi - 1.0) * g - e2 * lap_m(g, h, zp)
    cf2_per_kappa = cf2_of(_with(p, kappa=1.0))
    kappabar = float(np.sum(cf2_per_kappa * inner * mubar))
    sigmabar = float(np.sum((C_A / p.eps) * g * mubar))
    gammabar = float(np.sum(-lphi * mubar))
    return phibar, kappabar, sigmabar, gammabar


def _with(p, **kw):
    import dataclasses
    return dataclasses.replace(p, **kw)


def flow_vjp(phi, mu, psibar, p, omegabar=None, shift=0.0):
    """Adjoint of psi(phi, mu) (source, vorticity solve, stream solve).

    omegabar_total = omegabar - L^-1 psibar (omegabar: the adjoint of omega
    from the next step's backward-Euler vorticity update, inertial variant),
    fbar = (L - shift)^-1 omegabar_total, then the cross product
    f = (D_m phi x D_m mu) / eta.  Returns (phibar, mubar, omegabar_prev)
    with omegabar_prev = -shift fbar, the adjoint passed to the previous
    vorticity (zero for the Stokes step, shift = 0)."""
    h, zp = p.h, p.z_periodic
    per = (True, False, zp)
    fbar = []
    for c in range(3):
        ob = -solve_poisson(psibar[c], h, per)
        if omegabar is not None:
            ob = ob + omegabar[c]
        fbar.append(solve_poisson(ob, h, per, shift))
    a = grad(pad_mirror(phi, 1, zp), h)
    b = grad(pad_mirror(mu, 1, zp), h)
    ie = 1.0 / p.eta
    abar = [(b[1] * fbar[2] - b[2] * fbar[1]) * ie,      # (b x fbar) / eta
            (b[2] * fbar[0] - b[0] * fbar[2]) * ie,
            (b[0] * fbar[1] - b[1] * fbar[0]) * ie]
    bbar = [(fbar[1] * a[2] - fbar[2] * a[1]) * ie,      # (fbar x a) / eta
            (fbar[2] * a[0] - fbar[0] * a[2]) * ie,
            (fbar[0] * a[1] - fbar[1] * a[0]) * ie]
    return (grad_mirror_t(abar, h, zp), grad_mirror_t(bbar, h, zp),
            [-shift * fbar[c] for c in range(3)])


def update_vjp(phi, vel, phibar_next, p, dt):
    """Adjoint of phi^{n+1} = phi^n + dt [M (L_m mu^n + lambda^n) - v^n . D_m
    phi^n] for the adjoint phibar_next of phi^{n+1}.  Returns (phibar,
    mubar, psibar, V0bar): the adjoints of phi^n (through this update and
    lambda^n), mu^n, psi^n, and the contribution to the constant V0."""
    h, zp = p.h, p.z_periodic
    u = phibar_next
    lambar = dt * p.mobility * float(np.sum(u))
    phibar = u - dt * grad_mirror_t([vel[a] * u for a in range(3)], h, zp)
    phibar = phibar + lambar * p.k_vol * (-0.5 * h ** 3)
    mubar = dt * p.mobility * lap_m(u, h, zp)
    d = grad(pad_mirror(phi, 1, zp), h)
    vbar = [-dt * u * d[a] for a in range(3)]
    psibar = curl_zero(vbar, h, zp)
    return phibar, mubar, psibar, -lambar * p.k_vol


# ---------------------------------------------------------------- trajectory
def forward(p, phi0, dt, nsteps):
    """States 0..N of the forward oracle: phi, mu, gamma_A and the velocity."""
    st = init_state(p, phi0)
    traj = [dict(phi=st.phi, mu=st.mu, gamma=0.0, vel=velocity(st))]
    for _ in range(nsteps):
        step(st, dt)
        traj.append(dict(phi=st.phi, mu=st.mu, gamma=st.gamma_a, vel=velocity(st)))
    return traj


def loss(phi, target, h):
    return 0.5 * h ** 3 * float(np.sum((phi - target) ** 2))


def gradient(p, phi0, dt, nsteps, target=None, phibar_final=None):
    """Gradient of J (or of <phibar_final, phi^N> when given) with respect
    to phi^0, kappa and sigma.  Returns (J, phi0bar, kappabar, sigmabar)."""
    traj = forward(p, phi0, dt, nsteps)
    h = p.h
    phiN = traj[-1]["phi"]
    if phibar_final is None:
        J = loss(phiN, target, h)
        phibar = h ** 3 * (phiN - target)
    else:
        J = float(np.sum(phibar_final * phiN))
        phibar = np.array(phibar_final, dtype=np.float64, copy=True)
    mubar = np.zeros_like(phibar)
    psibar = [np.zeros_like(phibar) for _ in range(3)]
    omegabar = [np.zeros_like(phibar) for _ in range(3)]
    shift = inertial_shift(p, dt)   # 0 for the Stokes step
    kb = sb = v0b = a0b = 0.0
    cg = p.k_area * 3.0 * p.eps / (2.0 * math.sqrt(2.0))
    for n in range(nsteps - 1, -1, -1):
        s1 = traj[n + 1]
        fp, fm, omegabar = flow_vjp(s1["phi"], s1["mu"], psibar, p, omegabar, shift)
        phibar = phibar + fp
        mubar = mubar + fm
        dp, dk, ds, dg = mu_vjp(s1["phi"], s1["gamma"], mubar, p)
        phibar = phibar + dp
        kb += dk
        sb += ds
        if p.fe_kind == HELFRICH and cg != 0.0:
            phibar = phibar + dg * cg * area_grad(s1["phi"], p)
            a0b -= dg * cg
        s0 = traj[n]
        phibar, mubar, psibar, dv = update_vjp(s0["phi"], s0["vel"], phibar, p, dt)
        v0b += dv
    s0 = traj[0]   # the initial vorticity is the Stokes one of phi^0
    fp, fm, _ = flow_vjp(s0["phi"], s0["mu"], psibar, p, omegabar, 0.0)
    phibar = phibar + fp
    mubar = mubar + fm
    dp, dk, ds, _ = mu_vjp(s0["phi"], 0.0, mubar, p)
    phibar = phibar + dp + v0b * (-0.5 * h ** 3)
    if p.fe_kind == HELFRICH and a0b != 0.0:
        phibar = phibar + a0b * area_grad(s0["phi"], p)
    return J, phibar, kb + dk, sb + ds
