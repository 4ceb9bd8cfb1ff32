"""Uniform cubic grid and finite-difference operators (oracle, FP64).

Numerical-implementation section: a fixed cubic grid with equal spacing in
x, y, z and standard finite differences.  Readings fixed here:

* cells are indexed [k][j][i] (z, y, x); x is the periodic flow axis
  (boundary-conditions section: periodic in the flow direction);
* flow fields (omega, psi) carry Dirichlet data on the ghost nodes j = -1 and
  j = n of each walled axis -- the walls themselves -- taken from the
  body-free flow (boundary-conditions section);
* scalar fields (phi, mu, g) use an even mirror about the cell face next to
  the wall (no-flux), index -1-m <-> m;
* the Laplacian is the 7-point stencil, first derivatives are central
  differences, curl is built from the central differences.

Pinned by: eigenvector of the Dirichlet/periodic 7-point operator
(sin/cos products), Couette and planar-Poiseuille closed forms (curl and
Laplacian of polynomials), discrete divergence of a curl vanishing to
round-off, pure-loop transcription on tiny grids.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class GridSpec:
    nx: int
    ny: int
    nz: int
    h: float = 1.0
    z_periodic: bool = False   # y is always walled, x always periodic

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz


def pad_flow(u: np.ndarray, ghost_yz: np.ndarray, z_periodic: bool) -> np.ndarray:
    """One ghost layer for a flow component.

    ``ghost_yz`` has shape (nz + 2, ny + 2): entry [k + 1, j + 1] is the
    Dirichlet value on the wall node (j or k equal to -1 or n); it is
    independent of x because every channel flow here is x-invariant.
    Edge and corner ghosts are never read by the 7-point or central stencils
    and are left as NaN so that a stray read would show.
    """
    nz, ny, nx = u.shape
    P = np.full((nz + 2, ny + 2, nx + 2), np.nan)
    P[1:-1, 1:-1, 1:-1] = u
    P[1:-1, 1:-1, 0] = u[:, :, -1]
    P[1:-1, 1:-1, -1] = u[:, :, 0]
    P[1:-1, 0, 1:-1] = ghost_yz[1:-1, 0][:, None]
    P[1:-1, -1, 1:-1] = ghost_yz[1:-1, -1][:, None]
    if z_periodic:
        P[0, 1:-1, 1:-1] = u[-1]
        P[-1, 1:-1, 1:-1] = u[0]
    else:
        P[0, 1:-1, 1:-1] = ghost_yz[0, 1:-1][:, None]
        P[-1, 1:-1, 1:-1] = ghost_yz[-1, 1:-1][:, None]
    return P


def pad_homogeneous(u: np.ndarray, periodic: tuple) -> np.ndarray:
    """One ghost layer with zero Dirichlet data or periodic wrap per axis.

    ``periodic`` = (px, py, pz) booleans.  Used by the standalone Poisson
    operator.
    """
    nz, ny, nx = u.shape
    P = np.full((nz + 2, ny + 2, nx + 2), np.nan)
    P[1:-1, 1:-1, 1:-1] = u
    px, py, pz = periodic
    if px:
        P[1:-1, 1:-1, 0], P[1:-1, 1:-1, -1] = u[:, :, -1], u[:, :, 0]
    else:
        P[1:-1, 1:-1, 0] = P[1:-1, 1:-1, -1] = 0.0
    if py:
        P[1:-1, 0, 1:-1], P[1:-1, -1, 1:-1] = u[:, -1, :], u[:, 0, :]
    else:
        P[1:-1, 0, 1:-1] = P[1:-1, -1, 1:-1] = 0.0
    if pz:
        P[0, 1:-1, 1:-1], P[-1, 1:-1, 1:-1] = u[-1], u[0]
    else:
        P[0, 1:-1, 1:-1] = P[-1, 1:-1, 1:-1] = 0.0
    return P


def pad_mirror(u: np.ndarray, width: int, z_periodic: bool) -> np.ndarray:
    """``width`` ghost layers for a scalar: periodic in x, even mirror about
    the wall face in y, mirror or periodic in z (numpy 'symmetric' mode is
    exactly the face mirror: index -1-m takes the value of index m)."""
    w = width
    P = np.pad(u, ((0, 0), (0, 0), (w, w)), mode="wrap")
    P = np.pad(P, ((0, 0), (w, w), (0, 0)), mode="symmetric")
    P = np.pad(P, ((w, w), (0, 0), (0, 0)), mode="wrap" if z_periodic else "symmetric")
    return P


def lap(P: np.ndarray, h: float) -> np.ndarray:
    """7-point Laplacian of the interior of a 1-ghost padded array."""
    c = P[1:-1, 1:-1, 1:-1]
    s = (P[1:-1, 1:-1, 2:] + P[1:-1, 1:-1, :-2]
         + P[1:-1, 2:, 1:-1] + P[1:-1, :-2, 1:-1]
         + P[2:, 1:-1, 1:-1] + P[:-2, 1:-1, 1:-1])
    return (s - 6.0 * c) / (h * h)


def grad(P: np.ndarray, h: float):
    """Central first differences (d/dx, d/dy, d/dz) of a 1-ghost padded array."""
    inv2h = 1.0 / (2.0 * h)
    gx = (P[1:-1, 1:-1, 2:] - P[1:-1, 1:-1, :-2]) * inv2h
    gy = (P[1:-1, 2:, 1:-1] - P[1:-1, :-2, 1:-1]) * inv2h
    gz = (P[2:, 1:-1, 1:-1] - P[:-2, 1:-1, 1:-1]) * inv2h
    return gx, gy, gz


def lap_mirror(u: np.ndarray, h: float, z_periodic: bool) -> np.ndarray:
    return lap(pad_mirror(u, 1, z_periodic), h)


def grad_mirror(u: np.ndarray, h: float, z_periodic: bool):
    return grad(pad_mirror(u, 1, z_periodic), h)


def curl(psi, ghosts, h: float, z_periodic: bool):
    """v = curl psi with central differences (main-text eq. vecpot).

    ``psi`` = (psi_x, psi_y, psi_z) cell fields, ``ghosts`` = their wall-node
    Dirichlet data (each (nz + 2, ny + 2)).
    """
    gx = [grad(pad_flow(psi[c], ghosts[c], z_periodic), h) for c in range(3)]
    # gx[c][a] = d psi_c / d x_a
    vx = gx[2][1] - gx[1][2]
    vy = gx[0][2] - gx[2][0]
    vz = gx[1][0] - gx[0][1]
    return vx, vy, vz
