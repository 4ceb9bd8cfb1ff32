"""Second, independently written transcription of one step with plain Python
loops (tiny grids only; oracle test infrastructure).

It re-derives every index by hand -- periodic wrap with ``%``, the wall
mirror with an explicit reflection function, Dirichlet wall nodes looked up
from the wall data -- and solves the Poisson problems with a dense matrix
assembled cell by cell.  Agreement with the vectorised oracle to round-off
pins the vectorised padding / slicing (main-text eqs. gen2, gen1, gen3 and
the segregated order of the numerical-implementation section).
"""
from __future__ import annotations

import math

import numpy as np

from inputs import CAHN_HILLIARD


def _mirror(j, n):
    """Face mirror: index -1-m -> m, n+m -> n-1-m."""
    if j < 0:
        return -1 - j
    if j >= n:
        return 2 * n - 1 - j
    return j


class _Scalar:
    """Cell field with periodic x, mirrored y, mirrored or periodic z."""

    def __init__(self, a, zper):
        self.a, self.zper = a, zper
        self.nz, self.ny, self.nx = a.shape

    def __call__(self, k, j, i):
        i %= self.nx
        j = _mirror(j, self.ny)
        k = k % self.nz if self.zper else _mirror(k, self.nz)
        return self.a[k, j, i]


class _Flow:
    """Cell field with periodic x, wall-node data on walled axes."""

    def __init__(self, a, ring, zper):
        self.a, self.ring, self.zper = a, ring, zper
        self.nz, self.ny, self.nx = a.shape

    def __call__(self, k, j, i):
        i %= self.nx
        if self.zper:
            k %= self.nz
        if j < 0 or j >= self.ny or k < 0 or k >= self.nz:
            return self.ring[k + 1, j + 1]
        return self.a[k, j, i]


def _lap_at(F, k, j, i, h):
    c = F(k, j, i)
    return (F(k, j, i + 1) + F(k, j, i - 1) + F(k, j + 1, i) + F(k, j - 1, i)
            + F(k + 1, j, i) + F(k - 1, j, i) - 6.0 * c) / (h * h)


def _grad_at(F, k, j, i, h):
    return ((F(k, j, i + 1) - F(k, j, i - 1)) / (2 * h),
            (F(k, j + 1, i) - F(k, j - 1, i)) / (2 * h),
            (F(k + 1, j, i) - F(k - 1, j, i)) / (2 * h))


def _cells(shape):
    nz, ny, nx = shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                yield k, j, i


def _mu_field(phi, p, gamma_a):
    shape = phi.shape
    P = _Scalar(phi, p.z_periodic)
    if p.fe_kind == CAHN_HILLIARD:
        out = np.empty(shape)
        for k, j, i in _cells(shape):
            f = phi[k, j, i]
            out[k, j, i] = f ** 3 - f - p.sigma * _lap_at(P, k, j, i, p.h)
        return out
    g = np.empty(shape)
    for k, j, i in _cells(shape):
        f = phi[k, j, i]
        g[k, j, i] = f ** 3 - f - p.eps ** 2 * _lap_at(P, k, j, i, p.h)
    Gf = _Scalar(g, p.z_periodic)
    cf = 3.0 * math.sqrt(2.0) * p.kappa / (8.0 * p.eps ** 3)
    out = np.empty(shape)
    for k, j, i in _cells(shape):
        f = phi[k, j, i]
        out[k, j, i] = (2.0 * cf * ((3 * f * f - 1) * g[k, j, i] - p.eps ** 2 * _lap_at(Gf, k, j, i, p.h))
                        - gamma_a * _lap_at(P, k, j, i, p.h))
        # membrane tension sigma: derivative of sigma times the face area
        out[k, j, i] += p.sigma * 3.0 / (2.0 * math.sqrt(2.0) * p.eps) * g[k, j, i]
    return out


def _dense_solve(f, ring, p):
    """Assemble lap u = f cell by cell (wall data moved to the rhs) and solve."""
    nz, ny, nx = f.shape
    n = nx * ny * nz
    idx = lambda k, j, i: (k * ny + j) * nx + i
    M = np.zeros((n, n))
    b = np.zeros(n)
    h2 = p.h * p.h
    for k, j, i in _cells(f.shape):
        r = idx(k, j, i)
        b[r] = f[k, j, i]
        M[r, r] -= 6.0 / h2
        for dk, dj, di in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
            kk, jj, ii = k + dk, j + dj, (i + di) % nx
            if p.z_periodic:
                kk %= nz
            if 0 <= jj < ny and 0 <= kk < nz:
                M[r, idx(kk, jj, ii)] += 1.0 / h2
            else:
                b[r] -= ring[kk + 1, jj + 1] / h2
    return np.linalg.solve(M, b).reshape(f.shape)


def brute_step(phi, mu, psi, V, V0, A0, p, bf, dt):
    """One step (same readings as ``oracle.step``) with loops; returns
    (phi, mu, omega, psi, V_new, A_new)."""
    shape = phi.shape
    h = p.h
    zp = p.z_periodic
    P, Mu = _Scalar(phi, zp), _Scalar(mu, zp)
    Ps = [_Flow(psi[c], bf.psi_b[c], zp) for c in range(3)]
    lam_v = p.k_vol * (V - V0)
    phi_new = np.empty(shape)
    for k, j, i in _cells(shape):
        d = [_grad_at(Ps[c], k, j, i, h) for c in range(3)]  # d[c][a] = d psi_c / d x_a
        vx = d[2][1] - d[1][2]
        vy = d[0][2] - d[2][0]
        vz = d[1][0] - d[0][1]
        gx, gy, gz = _grad_at(P, k, j, i, h)
        rate = p.mobility * (_lap_at(Mu, k, j, i, h) + lam_v) - (vx * gx + vy * gy + vz * gz)
        phi_new[k, j, i] = phi[k, j, i] + dt * rate
    Pn = _Scalar(phi_new, zp)
    V_new = 0.0
    A_new = 0.0
    c_a = 3.0 / (2.0 * math.sqrt(2.0))
    for k, j, i in _cells(shape):
        f = phi_new[k, j, i]
        V_new += 0.5 * (1.0 - f) * h ** 3
        gx, gy, gz = _grad_at(Pn, k, j, i, h)
        A_new += c_a * (0.5 * p.eps * (gx * gx + gy * gy + gz * gz)
                        + (f * f - 1) ** 2 / (4 * p.eps)) * h ** 3
    gamma_a = p.k_area * (A_new - A0) * 3.0 * p.eps / (2.0 * math.sqrt(2.0))
    mu_new = _mu_field(phi_new, p, gamma_a)
    Mn = _Scalar(mu_new, zp)
    f = [np.empty(shape) for _ in range(3)]
    for k, j, i in _cells(shape):
        a = _grad_at(Pn, k, j, i, h)
        b = _grad_at(Mn, k, j, i, h)
        f[0][k, j, i] = (a[1] * b[2] - a[2] * b[1]) / p.eta
        f[1][k, j, i] = (a[2] * b[0] - a[0] * b[2]) / p.eta
        f[2][k, j, i] = (a[0] * b[1] - a[1] * b[0]) / p.eta
    omega = [_dense_solve(f[c], bf.omega_b[c], p) for c in range(3)]
    psi_new = [_dense_solve(-omega[c], bf.psi_b[c], p) for c in range(3)]
    return phi_new, mu_new, omega, psi_new, V_new, A_new
