"""Body-free channel flows that supply the wall data (oracle, FP64).

Boundary-conditions section: no-slip walls; the Dirichlet data for omega and
psi on the walls are those of the flow without bodies, obtained from an
analytic expression or, when there is none, from a numerical solver.  The
flow direction is periodic.  Readings (x is the flow axis; walls sit on the
ghost nodes, coordinate y = (j + 1) h, height H = (n + 1) h):

* Couette (walls at y only, z periodic; the paper's eq. BCsCouete is garbled,
  so the data are derived from the velocity it states): v_x = v_lo +
  (v_hi - v_lo) y / H, psi = (0, 0, v_lo y + (v_hi - v_lo) y^2 / (2H)),
  omega = (0, 0, -(v_hi - v_lo) / H).
* Planar Poiseuille (walls at y, z periodic): v_x = 4 U y (H - y) / H^2,
  psi_z = 4 U (H y^2/2 - y^3/3) / H^2, omega_z = -4 U (H - 2y) / H^2.
* Rectangular duct (walls at y and z; the paper gives only the cylinder):
  the numerical route of the boundary-conditions section, done on the grid.
  u0 solves the 2-D discrete problem lap u0 = -1 with u0 = 0 on the wall
  nodes and is scaled so that its maximum over the cells is U; chi solves
  lap chi = u0 with chi = 0 on the wall nodes; then v = curl psi and
  omega = curl v for psi = (0, -d chi/dz, d chi/dy), so the wall data are
  omega = (0, du0/dz, -du0/dy) and psi = (0, -dchi/dz, dchi/dy), with the
  normal derivative on a wall node taken by the second-order one-sided
  difference (-3 f_w + 4 f_1 - f_2) / (2h) and the tangential one zero
  (u0 and chi vanish along the wall).
* Quiescent: walls at y and z, all data zero.

Pinned by: Couette and planar-Poiseuille body-free steps reproduce the
closed forms to round-off; the duct velocity converges at second order to
the textbook series solution; velocity vanishes at the walls.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from inputs import COUETTE, POISEUILLE_DUCT, POISEUILLE_PLANAR, QUIESCENT
from .poisson import solve_poisson, solve_flow_component


@dataclass
class BaseFlow:
    kind: int
    z_periodic: bool
    omega_b: list      # 3 arrays (nz + 2, ny + 2): wall-node data of omega
    psi_b: list        # 3 arrays: wall-node data of psi
    vel_b: list        # 3 arrays: wall velocity (no-slip) on the wall nodes


def _ring(ny, nz):
    return np.full((nz + 2, ny + 2), np.nan)


def _node_coord(n, h):
    """Coordinates of nodes -1 .. n along a walled axis (walls at 0, H)."""
    return (np.arange(-1, n + 1, dtype=np.float64) + 1.0) * h


def _solve_2d(rhs2d, h):
    """Solve the x-invariant problem on a (nz, ny) section, zero wall data."""
    nz, ny = rhs2d.shape
    return solve_poisson(rhs2d[:, :, None], h, (True, False, False))[:, :, 0]


def duct_profile(ny, nz, h, u_max):
    """u0 and chi of the duct reading (module docstring); (nz, ny) arrays."""
    u0 = _solve_2d(-np.ones((nz, ny)), h)
    u0 *= u_max / u0.max()
    chi = _solve_2d(u0, h)
    return u0, chi


def _one_sided(first, second, h):
    """d f / dn at a wall node where f = 0, f_1 = first, f_2 = second
    (n pointing into the channel)."""
    return (4.0 * first - second) / (2.0 * h)


def base_flow(kind: int, nx: int, ny: int, nz: int, h: float, u_max=0.0, v_lo=0.0,
              v_hi=0.0) -> BaseFlow:
    zper = kind in (COUETTE, POISEUILLE_PLANAR)
    om = [_ring(ny, nz) for _ in range(3)]
    ps = [_ring(ny, nz) for _ in range(3)]
    vw = [_ring(ny, nz) for _ in range(3)]
    for arrs in (om, ps, vw):
        for a in arrs:
            a[:, 0] = a[:, -1] = 0.0
            a[0, :] = a[-1, :] = 0.0
    yn = _node_coord(ny, h)
    H = (ny + 1) * h
    if kind == COUETTE:
        psi_z = v_lo * yn + (v_hi - v_lo) * yn ** 2 / (2.0 * H)
        om_z = -(v_hi - v_lo) / H
        for side, jj in ((0, 0), (1, ny + 1)):
            ps[2][:, jj] = psi_z[jj]
            om[2][:, jj] = om_z
            vw[0][:, jj] = v_lo if side == 0 else v_hi
    elif kind == POISEUILLE_PLANAR:
        U = u_max
        psi_z = 4.0 * U * (H * yn ** 2 / 2.0 - yn ** 3 / 3.0) / H ** 2
        om_z = -4.0 * U * (H - 2.0 * yn) / H ** 2
        for jj in (0, ny + 1):
            ps[2][:, jj] = psi_z[jj]
            om[2][:, jj] = om_z[jj]
    elif kind == POISEUILLE_DUCT:
        u0, chi = duct_profile(ny, nz, h, u_max)
        # y walls (j = -1 and j = ny), k = 0 .. nz-1
        d_u_lo = _one_sided(u0[:, 0], u0[:, 1], h)          # du/dy at y = 0
        d_u_hi = -_one_sided(u0[:, -1], u0[:, -2], h)       # du/dy at y = H
        d_c_lo = _one_sided(chi[:, 0], chi[:, 1], h)
        d_c_hi = -_one_sided(chi[:, -1], chi[:, -2], h)
        om[2][1:-1, 0], om[2][1:-1, -1] = -d_u_lo, -d_u_hi   # omega_z = -du/dy
        ps[2][1:-1, 0], ps[2][1:-1, -1] = d_c_lo, d_c_hi     # psi_z = dchi/dy
        # z walls (k = -1 and k = nz), j = 0 .. ny-1
        e_u_lo = _one_sided(u0[0, :], u0[1, :], h)          # du/dz at z = 0
        e_u_hi = -_one_sided(u0[-1, :], u0[-2, :], h)
        e_c_lo = _one_sided(chi[0, :], chi[1, :], h)
        e_c_hi = -_one_sided(chi[-1, :], chi[-2, :], h)
        om[1][0, 1:-1], om[1][-1, 1:-1] = e_u_lo, e_u_hi     # omega_y = du/dz
        ps[1][0, 1:-1], ps[1][-1, 1:-1] = -e_c_lo, -e_c_hi   # psi_y = -dchi/dz
    elif kind == QUIESCENT:
        pass
    else:
        raise ValueError(f"unknown flow kind {kind}")
    return BaseFlow(kind=kind, z_periodic=zper, omega_b=om, psi_b=ps, vel_b=vw)


def body_free_fields(bf: BaseFlow, nx: int, ny: int, nz: int, h: float):
    """The discrete flow with no body: lap omega0 = 0, lap psi0 = -omega0
    with the wall data of ``bf`` (results section: omega_0, xi_0 are the
    fields in the absence of the object).  Returns (omega0, psi0), each a
    list of three [nz][ny][nx] arrays (x-invariant)."""
    zero = np.zeros((nz, ny, nx))
    om0 = [solve_flow_component(zero, bf.omega_b[c], h, bf.z_periodic) for c in range(3)]
    ps0 = [solve_flow_component(-om0[c], bf.psi_b[c], h, bf.z_periodic) for c in range(3)]
    return om0, ps0
