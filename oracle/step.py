"""One time step of the vorticity--stream-vector phase-field method (oracle).

Main-text eqs. gen2, gen1, gen3 (SM eq. 29) advanced as in the
numerical-implementation section: forward Euler for phi, then the
vorticity Poisson problem, then the stream-vector Poisson problem, all in the
same step with the same dt.  Step n -> n+1:

  1. v^n = curl psi^n                                   (eq. vecpot)
  2. lambda_V^n = K_V (V[phi^n] - V0)                   (SM eqs. 37-38)
  3. phi^{n+1} = phi^n + dt [M (lap mu^n + lambda_V^n) - v^n . grad phi^n]
  4. gamma_A^{n+1} = K_A (A[phi^{n+1}] - A0) 3 eps / (2 sqrt 2)
  5. mu^{n+1} = mu(phi^{n+1}; gamma_A^{n+1})            (eq. 31 / SM eq. 35)
  6. f = grad phi^{n+1} x grad mu^{n+1} / eta           (eq. gen1)
  7. omega^{n+1}: lap omega = f, wall data omega_b      (eq. gen1)
  8. psi^{n+1}:   lap psi = -omega^{n+1}, wall data psi_b (eq. gen3)

Readings: the vorticity source uses the new mu (the flow is instantaneous
Stokes for the current interface); advection uses the velocity of the
previous stream vector, as the segregated order implies; the initial state
solves 5-8 for phi^0 with gamma_A = 0 (A = A0).

Time-dependent walls (supplementary material, the time-dependency
paragraph after eq. 36: a flow that speeds up, slows down or oscillates
changes only the boundary conditions, not the system of equations).  With
``wall_motion`` set, each wall speed of the body-free flow becomes
s(t) = s0 + ramp t + amplitude sin(2 pi frequency t + phase): index 0 is the
Couette wall at y = 0 or the Poiseuille speed U, index 1 the Couette wall at
y = H.  Step n -> n+1 advects phi with the flow of time t^n (its wall data
are those of t^n) and solves steps 7-8 with the wall data of t^{n+1}.

Inertial variant (SM eq. 36, density rho > 0): the vorticity obeys
(rho / eta) d omega / dt - lap omega = -f, a heat equation.  Reading: one
backward-Euler step per time step, so step 7 becomes

  7'. (lap - s) omega^{n+1} = f - s omega^n,  s = rho / (eta dt),

with the same wall data; phi and psi are unchanged.  The initial vorticity
is the non-inertial (Stokes) solution for phi^0.  rho = 0 is eq. gen1.

Pinned by the module pins of grid / poisson / flow / free_energy, by the
Couette and Poiseuille body-free steady states, by the closed-form profiles
of oscillating and ramped walls at every step and the exact base-flow
difference one moving-wall step makes with a body present, by the closed-form
advection of a sine profile, by the free-energy dissipation identity and by a
pure-loop transcription of the whole step on a tiny grid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .grid import pad_mirror, lap, grad, curl
from .poisson import solve_flow_component
from .flow import base_flow, BaseFlow
from .free_energy import (chem_potential, volume, area, area_multiplier,
                          volume_multiplier)


@dataclass
class OracleParams:
    nx: int
    ny: int
    nz: int
    h: float
    flow_kind: int
    u_max: float
    v_lo: float
    v_hi: float
    eta: float
    fe_kind: int
    sigma: float
    kappa: float
    eps: float
    mobility: float
    k_area: float
    k_vol: float
    mu_prefactor_half: bool = False
    rho: float = 0.0            # fluid density; > 0 selects SM eq. 36
    # time-dependent walls: (ramp, amplitude, frequency, phase), each a pair
    # (wall 0, wall 1); None for steady walls
    wall_motion: tuple = None

    @property
    def z_periodic(self):
        from inputs import COUETTE, POISEUILLE_PLANAR
        return self.flow_kind in (COUETTE, POISEUILLE_PLANAR)


def params_from_workload(w) -> OracleParams:
    return OracleParams(nx=w.nx, ny=w.ny, nz=w.nz, h=w.h, flow_kind=w.flow_kind,
                        u_max=w.u_max, v_lo=w.v_lo, v_hi=w.v_hi, eta=w.eta,
                        fe_kind=w.fe_kind, sigma=w.sigma, kappa=w.kappa, eps=w.eps,
                        mobility=w.mobility, k_area=w.k_area, k_vol=w.k_vol,
                        rho=getattr(w, "rho", 0.0),
                        wall_motion=getattr(w, "wall_motion", None))


@dataclass
class OracleState:
    p: OracleParams
    bf: BaseFlow
    phi: np.ndarray
    mu: np.ndarray
    omega: list
    psi: list
    V0: float
    A0: float
    V: float
    A: float
    gamma_a: float
    lambda_v: float = 0.0
    t: float = 0.0
    nstep: int = 0
    extra: dict = field(default_factory=dict)


def velocity(st: OracleState):
    return curl(st.psi, st.bf.psi_b, st.p.h, st.p.z_periodic)


def _mu(phi, p, gamma_a):
    return chem_potential(phi, p.fe_kind, p.h, p.z_periodic, sigma=p.sigma, kappa=p.kappa,
                          eps=p.eps, gamma_a=gamma_a, mu_prefactor_half=p.mu_prefactor_half)


def vorticity_source(phi, mu, p):
    zp = p.z_periodic
    gp = grad(pad_mirror(phi, 1, zp), p.h)
    gm = grad(pad_mirror(mu, 1, zp), p.h)
    inv_eta = 1.0 / p.eta
    fx = (gp[1] * gm[2] - gp[2] * gm[1]) * inv_eta
    fy = (gp[2] * gm[0] - gp[0] * gm[2]) * inv_eta
    fz = (gp[0] * gm[1] - gp[1] * gm[0]) * inv_eta
    return [fx, fy, fz]


def inertial_shift(p, dt) -> float:
    """s = rho / (eta dt) of the backward-Euler vorticity step (0: Stokes)."""
    return p.rho / (p.eta * dt) if p.rho > 0.0 else 0.0


def flow_solve(phi, mu, p, bf, omega_prev=None, dt=None):
    """Steps 6-8: source, vorticity and stream-vector solves.  With
    omega_prev and p.rho > 0 the vorticity solve is the backward-Euler step
    7' of the inertial variant."""
    f = vorticity_source(phi, mu, p)
    s = inertial_shift(p, dt) if omega_prev is not None else 0.0
    if s > 0.0:
        omega = [solve_flow_component(f[c] - s * omega_prev[c], bf.omega_b[c], p.h,
                                      p.z_periodic, shift=s) for c in range(3)]
    else:
        omega = [solve_flow_component(f[c], bf.omega_b[c], p.h, p.z_periodic) for c in range(3)]
    psi = [solve_flow_component(-omega[c], bf.psi_b[c], p.h, p.z_periodic) for c in range(3)]
    return omega, psi


def wall_speeds(p: OracleParams, t: float):
    """(u_max, v_lo, v_hi) of the body-free flow at time t: the steady values,
    or with ``wall_motion`` s(t) = s0 + ramp t + amplitude sin(2 pi f t + phase)
    (wall 0: v_lo, or u_max for Poiseuille; wall 1: v_hi)."""
    if p.wall_motion is None:
        return p.u_max, p.v_lo, p.v_hi
    ramp, amp, freq, phase = p.wall_motion

    def s(w, s0):
        return s0 + ramp[w] * t + amp[w] * np.sin(2.0 * np.pi * freq[w] * t + phase[w])
    from inputs import COUETTE
    if p.flow_kind == COUETTE:
        return p.u_max, s(0, p.v_lo), s(1, p.v_hi)
    return s(0, p.u_max), p.v_lo, p.v_hi


def base_flow_at(p: OracleParams, t: float) -> BaseFlow:
    """The body-free flow's wall data at time t (steady walls: any t)."""
    u, vlo, vhi = wall_speeds(p, t)
    return base_flow(p.flow_kind, p.nx, p.ny, p.nz, p.h, u_max=u, v_lo=vlo, v_hi=vhi)


def init_state(p: OracleParams, phi0: np.ndarray) -> OracleState:
    if p.wall_motion is not None and p.rho > 0.0:
        raise ValueError("time-dependent walls are provided for the non-inertial flow only")
    bf = base_flow_at(p, 0.0)
    phi = np.array(phi0, dtype=np.float64, copy=True)
    V0 = volume(phi, p.h)
    A0 = area(phi, p.eps, p.h, p.z_periodic)
    mu = _mu(phi, p, 0.0)
    omega, psi = flow_solve(phi, mu, p, bf)
    return OracleState(p=p, bf=bf, phi=phi, mu=mu, omega=omega, psi=psi, V0=V0, A0=A0,
                       V=V0, A=A0, gamma_a=0.0)


def phi_rate(st: OracleState, lambda_v: float):
    """Right-hand side of eq. gen2 at the current state."""
    p = st.p
    zp = p.z_periodic
    v = velocity(st)
    lap_mu = lap(pad_mirror(st.mu, 1, zp), p.h)
    gp = grad(pad_mirror(st.phi, 1, zp), p.h)
    adv = v[0] * gp[0] + v[1] * gp[1] + v[2] * gp[2]
    return p.mobility * (lap_mu + lambda_v) - adv


def step(st: OracleState, dt: float) -> OracleState:
    """Advance ``st`` in place by one step of size dt (module docstring)."""
    p = st.p
    lam_v = volume_multiplier(p.k_vol, st.V, st.V0)
    phi_new = st.phi + dt * phi_rate(st, lam_v)
    A_new = area(phi_new, p.eps, p.h, p.z_periodic)
    V_new = volume(phi_new, p.h)
    gamma_a = area_multiplier(p.k_area, A_new, st.A0, p.eps)
    mu_new = _mu(phi_new, p, gamma_a)
    if p.wall_motion is not None:      # wall data of t^{n+1} for the solves
        st.bf = base_flow_at(p, st.t + dt)
    omega, psi = flow_solve(phi_new, mu_new, p, st.bf, omega_prev=st.omega, dt=dt)
    st.phi, st.mu, st.omega, st.psi = phi_new, mu_new, omega, psi
    st.V, st.A, st.gamma_a, st.lambda_v = V_new, A_new, gamma_a, lam_v
    st.t += dt
    st.nstep += 1
    return st
