"""Exact discrete Poisson solves (oracle, FP64).

Main-text eqs. gen1 and gen3 are Poisson problems for each Cartesian
component; the numerical-implementation section only says they are solved
"using an iterative method".  The oracle does not iterate: it returns the
exact solution of the assembled 7-point system

    (L_h x)_c = sum_a (x_{c+e_a} + x_{c-e_a} - 2 x_c) / h^2 = b_c

with, per axis, periodic wrap or homogeneous Dirichlet data on the ghost
nodes -1 and n (inhomogeneous data are moved to the right-hand side by the
caller, see ``boundary_term``).  Two exact methods:

* ``solve_poisson_dense``: the assembled sparse matrix (``poisson_matrix``,
  a Kronecker sum of 1-D second-difference matrices) and a sparse direct
  solve -- the definition written out, used on small grids and as a pin;
* ``solve_poisson``: the exact eigen-decomposition of the same matrix.  The
  1-D Dirichlet matrix tridiag(1, -2, 1) of size n is diagonalised by the
  type-I sine transform, sin(pi (k+1) (j+1) / (n+1)) with eigenvalue
  2 cos(pi (k+1)/(n+1)) - 2; the periodic one by the discrete Fourier
  transform with eigenvalue 2 cos(2 pi k / n) - 2.

The inertial variant (SM eq. 36) needs the shifted operator L_h - s I
(s >= 0): the same two methods with every eigenvalue lowered by s, or the
matrix with s subtracted on the diagonal.

Pinned by: sin-product eigenvectors (closed form, with and without a
shift), agreement of the two methods, pure-loop assembly on tiny grids.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import pad_flow, pad_homogeneous, lap


def _second_difference_1d(n: int, periodic: bool) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(-2.0)
        for nb in (i - 1, i + 1):
            if 0 <= nb < n:
                rows.append(i); cols.append(nb); vals.append(1.0)
            elif periodic:
                rows.append(i); cols.append(nb % n); vals.append(1.0)
            # Dirichlet: the ghost node holds 0 and contributes nothing
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))  # duplicates summed


def poisson_matrix(shape, h: float, periodic) -> sp.csr_matrix:
    """Assembled 7-point operator for cells ordered [k][j][i] (x fastest)."""
    nz, ny, nx = shape
    px, py, pz = periodic
    Tx = _second_difference_1d(nx, px)
    Ty = _second_difference_1d(ny, py)
    Tz = _second_difference_1d(nz, pz)
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    L = (sp.kron(Tz, sp.kron(Iy, Ix)) + sp.kron(Iz, sp.kron(Ty, Ix))
         + sp.kron(Iz, sp.kron(Iy, Tx)))
    return (L / (h * h)).tocsr()


def apply_poisson(x: np.ndarray, h: float, periodic) -> np.ndarray:
    """L_h x with homogeneous Dirichlet / periodic ghosts (stencil form)."""
    return lap(pad_homogeneous(x, periodic), h)


def solve_poisson_dense(b: np.ndarray, h: float, periodic, shift: float = 0.0) -> np.ndarray:
    """(L_h - shift I) x = b by a sparse direct solve of the assembled matrix."""
    L = poisson_matrix(b.shape, h, periodic)
    if shift:
        L = L - shift * sp.identity(L.shape[0], format="csr")
    x = spla.spsolve(L.tocsc(), b.reshape(-1))
    return np.asarray(x).reshape(b.shape)


def _eigenvalues(n: int, h: float, periodic: bool) -> np.ndarray:
    k = np.arange(n, dtype=np.float64)
    if periodic:
        return (2.0 * np.cos(2.0 * np.pi * k / n) - 2.0) / (h * h)
    return (2.0 * np.cos(np.pi * (k + 1.0) / (n + 1.0)) - 2.0) / (h * h)


def solve_poisson(b: np.ndarray, h: float, periodic, shift: float = 0.0) -> np.ndarray:
    """Exact solve of (L_h - shift I) x = b by eigen-decomposition (see
    module docstring)."""
    nz, ny, nx = b.shape
    px, py, pz = periodic
    if px and py and pz and shift <= 0.0:
        raise ValueError("all-periodic Poisson problem is singular")
    X = np.array(b, dtype=np.float64, copy=True)
    dirichlet_axes = [ax for ax, per in ((2, px), (1, py), (0, pz)) if not per]
    periodic_axes = [ax for ax, per in ((2, px), (1, py), (0, pz)) if per]
    for ax in dirichlet_axes:
        X = sfft.dst(X, type=1, axis=ax)
    if periodic_axes:
        X = sfft.fftn(X, axes=periodic_axes)
    lam = (_eigenvalues(nz, h, pz)[:, None, None]
           + _eigenvalues(ny, h, py)[None, :, None]
           + _eigenvalues(nx, h, px)[None, None, :]) - shift
    X = X / lam
    if periodic_axes:
        X = sfft.ifftn(X, axes=periodic_axes).real
    for ax in dirichlet_axes:
        X = sfft.idst(X, type=1, axis=ax)
    return X


def boundary_term(ghost_yz: np.ndarray, shape, h: float, z_periodic: bool) -> np.ndarray:
    """Contribution of the wall-node data to L_h at the wall-adjacent cells,
    so that L_h u = f  <=>  L_h^0 u = f - boundary_term (L_h^0: zero ghosts)."""
    zero = np.zeros(shape)
    return lap(pad_flow(zero, ghost_yz, z_periodic), h)


def solve_flow_component(f: np.ndarray, ghost_yz: np.ndarray, h: float,
                         z_periodic: bool, shift: float = 0.0) -> np.ndarray:
    """Solve (L_h - shift I) u = f for one Cartesian component with Dirichlet
    wall data ``ghost_yz`` and periodic x (and z when ``z_periodic``).  The
    shift does not couple neighbours, so the wall data enter exactly as for
    L_h."""
    rhs = f - boundary_term(ghost_yz, f.shape, h, z_periodic)
    return solve_poisson(rhs, h, (True, False, z_periodic), shift)
