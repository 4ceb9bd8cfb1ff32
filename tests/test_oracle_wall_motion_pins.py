"""Pins of the oracle's time-dependent walls against closed forms.

The supplementary material's time-dependency paragraph (after eq. 36): a flow
that speeds up, slows down or oscillates needs no change to the system of
equations, only to its boundary conditions.  Since the flow is Stokes flow
(instantaneous), the body-free discrete fields at every step are the
closed-form profiles of that step's wall speeds, and with a body present the
moving walls add exactly the difference of the body-free fields.  No GPU.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from oracle.step import OracleParams, init_state, step, velocity, wall_speeds


def _params(nx, ny, nz, flow_kind, **kw):
    base = dict(nx=nx, ny=ny, nz=nz, h=1.0, flow_kind=flow_kind, u_max=0.0, v_lo=0.0,
                v_hi=0.0, eta=0.7, fe_kind=inputs.CAHN_HILLIARD, sigma=1.0, kappa=1.0, eps=1.0,
                mobility=1.0, k_area=0.0, k_vol=0.0)
    base.update(kw)
    return OracleParams(**base)


MOTION = ((0.3, -0.2), (0.02, 0.035), (40.0, 25.0), (0.4, -1.1))   # ramp, amp, freq, phase


def _s(s0, w, t):
    ramp, amp, freq, ph = MOTION
    return s0 + ramp[w] * t + amp[w] * math.sin(2 * math.pi * freq[w] * t + ph[w])


def test_wall_speeds_formula_and_steady_default():
    p = _params(6, 7, 4, inputs.COUETTE, v_lo=-0.05, v_hi=0.05, wall_motion=MOTION)
    for t in (0.0, 0.013, 0.2):
        u, lo, hi = wall_speeds(p, t)
        assert u == 0.0 and abs(lo - _s(-0.05, 0, t)) < 1e-15 and abs(hi - _s(0.05, 1, t)) < 1e-15
    q = _params(6, 7, 4, inputs.POISEUILLE_PLANAR, u_max=0.07, wall_motion=MOTION)
    u, lo, hi = wall_speeds(q, 0.05)
    assert abs(u - _s(0.07, 0, 0.05)) < 1e-15 and lo == 0.0 and hi == 0.0
    r = _params(6, 7, 4, inputs.COUETTE, v_lo=-0.05, v_hi=0.05)
    assert wall_speeds(r, 3.0) == (0.0, -0.05, 0.05)


def test_oscillating_couette_profile_at_every_step():
    """No body: after each step psi_z = v_lo(t) y + (v_hi(t) - v_lo(t)) y^2 /
    (2H), omega_z = -(v_hi(t) - v_lo(t)) / H and v_x = v_lo(t) + (v_hi(t) -
    v_lo(t)) y / H with the wall speeds of that step's time (walls on the
    ghost nodes, y = (j + 1) h, H = (ny + 1) h); phi does not move."""
    nx, ny, nz, dt = 6, 9, 4, 0.01
    p = _params(nx, ny, nz, inputs.COUETTE, v_lo=-0.05, v_hi=0.05, wall_motion=MOTION)
    st = init_state(p, np.ones((nz, ny, nx)))
    H = ny + 1.0
    y = np.arange(ny) + 1.0
    for n in range(6):
        t = n * dt
        lo, hi = _s(-0.05, 0, t), _s(0.05, 1, t)
        assert np.max(np.abs(st.psi[2] - (lo * y + (hi - lo) * y ** 2 / (2 * H))[None, :, None])) < 1e-13
        assert np.max(np.abs(st.omega[2] + (hi - lo) / H)) < 1e-14
        assert np.max(np.abs(velocity(st)[0] - (lo + (hi - lo) * y / H)[None, :, None])) < 1e-14
        for c in (0, 1):
            assert np.max(np.abs(st.psi[c])) < 1e-15
        step(st, dt)
        assert np.max(np.abs(st.phi - 1.0)) == 0.0
        assert abs(st.t - (n + 1) * dt) < 1e-15


def test_ramped_planar_poiseuille_profile_at_every_step():
    """No body, planar Poiseuille with U(t): psi_z = 4U(t)(H y^2/2 - y^3/3)/H^2
    and omega_z = -4U(t)(H - 2y)/H^2 exactly at every step."""
    nx, ny, nz, dt = 4, 11, 3, 0.02
    p = _params(nx, ny, nz, inputs.POISEUILLE_PLANAR, u_max=0.07, wall_motion=MOTION)
    st = init_state(p, np.ones((nz, ny, nx)))
    H = ny + 1.0
    y = np.arange(ny) + 1.0
    for n in range(5):
        U = _s(0.07, 0, n * dt)
        assert np.max(np.abs(st.psi[2] - (4 * U * (H * y ** 2 / 2 - y ** 3 / 3) / H ** 2)[None, :, None])) < 1e-13
        assert np.max(np.abs(st.omega[2] - (-4 * U * (H - 2 * y) / H ** 2)[None, :, None])) < 1e-14
        step(st, dt)


def test_moving_walls_add_the_base_flow_difference_with_a_body():
    """With a vesicle, one step with moving walls against the same step with
    steady walls at the speeds of t = 0: phi and mu agree (the phi update
    advects with the flow of t^0, the same in both), and the flow fields
    differ exactly by the body-free fields of the speed change,
    psi_z: dlo (y - y^2/(2H)) + dhi y^2/(2H), omega_z: -(dhi - dlo)/H."""
    dt = 1e-3
    w = inputs.vesicle(16, 9, 8, inputs.COUETTE, 0.9, 1.0, dt=dt, b_range=(0.3, 0.35))
    p0 = oracle.params_from_workload(w)
    p1 = oracle.params_from_workload(w)
    p1.wall_motion = MOTION
    p1.v_lo, p1.v_hi = p0.v_lo, p0.v_hi
    # steady walls at the moving walls' t = 0 speeds
    p0.v_lo, p0.v_hi = _s(p0.v_lo, 0, 0.0), _s(p0.v_hi, 1, 0.0)
    s0 = init_state(p0, w.phi0)
    s1 = init_state(p1, w.phi0)
    for c in range(3):
        assert np.max(np.abs(s0.psi[c] - s1.psi[c])) < 1e-15
    step(s0, dt)
    step(s1, dt)
    assert np.max(np.abs(s0.phi - s1.phi)) < 1e-15
    assert np.max(np.abs(s0.mu - s1.mu)) < 1e-14
    H = w.ny + 1.0
    y = (np.arange(w.ny) + 1.0)[None, :, None]
    dlo = _s(w.v_lo, 0, dt) - _s(w.v_lo, 0, 0.0)
    dhi = _s(w.v_hi, 1, dt) - _s(w.v_hi, 1, 0.0)
    dpsi = dlo * (y - y ** 2 / (2 * H)) + dhi * y ** 2 / (2 * H)
    assert np.max(np.abs((s1.psi[2] - s0.psi[2]) - dpsi)) < 1e-14
    assert np.max(np.abs((s1.omega[2] - s0.omega[2]) + (dhi - dlo) / H)) < 1e-14
    for c in (0, 1):
        assert np.max(np.abs(s1.psi[c] - s0.psi[c])) < 1e-14
        assert np.max(np.abs(s1.omega[c] - s0.omega[c])) < 1e-14


def test_moving_walls_rejected_with_inertia():
    p = _params(6, 7, 4, inputs.COUETTE, v_lo=-0.05, v_hi=0.05, wall_motion=MOTION, rho=1.0)
    with pytest.raises(ValueError):
        init_state(p, np.ones((4, 7, 6)))
