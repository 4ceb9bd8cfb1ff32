"""Thin convenience wrapper over the C ABI: allocates the device workspace
with torch, passes torch's current stream, marshals arrays.  All compute is
in libvsv.so."""
from __future__ import annotations

import numpy as np
import torch

from . import vsv as V

_DT = {np.float32: V.VSV_DTYPE_F32, np.float64: V.VSV_DTYPE_F64,
       torch.float32: V.VSV_DTYPE_F32, torch.float64: V.VSV_DTYPE_F64}


def _dtype_code(dt):
    if dt in _DT:
        return _DT[dt]
    return _DT[np.dtype(dt).type]


class Simulation:
    def __init__(self, nx, ny, nz, h=1.0, precision=V.VSV_MIXED, device="cuda:0", stream=None):
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz, self.h = nx, ny, nz, h
        self.precision = precision
        self.device = torch.device(device)
        nbytes = V.vsv_workspace_bytes(nx, ny, nz, precision)
        if nbytes == 0:
            raise ValueError("invalid grid shape")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.g = V.vsv_create(nx, ny, nz, h, precision, self._ws_ptr, nbytes,
                              self.stream.cuda_stream)

    # ------------------------------------------------------------ set-up
    @classmethod
    def from_workload(cls, w, precision=V.VSV_MIXED, solver=None, device="cuda:0", stream=None):
        s = cls(w.nx, w.ny, w.nz, w.h, precision, device, stream)
        s.configure(w, solver)
        return s

    def configure(self, w, solver=None):
        V.vsv_set_flow(self.g, w.flow_kind, w.u_max, w.v_lo, w.v_hi, w.eta, getattr(w, "rho", 0.0))
        V.vsv_set_free_energy(self.g, w.fe_kind, w.sigma, w.kappa, w.eps, w.mobility, w.k_area,
                              w.k_vol)
        if getattr(w, "wall_motion", None) is not None:
            V.vsv_set_wall_motion(self.g, w.wall_motion)
        if solver is not None:
            V.vsv_set_solver(self.g, solver)

    def solver_params(self):
        return V.vsv_default_solver(self.precision)

    def set_phi(self, phi, check=True):
        if isinstance(phi, torch.Tensor):
            t = phi.contiguous()
            return V.vsv_set_phi(self.g, t.data_ptr(), _dtype_code(t.dtype), int(t.is_cuda),
                                 check=check)
        a = np.ascontiguousarray(phi)
        return V.vsv_set_phi(self.g, a.ctypes.data, _dtype_code(a.dtype.type), 0, check=check)

    # ------------------------------------------------------------ run
    def step(self, nsteps, dt, check=True):
        return V.vsv_step(self.g, nsteps, dt, check=check)

    def field(self, fid, dtype=np.float64, on_device=False):
        if on_device:
            tdt = torch.float64 if dtype in (np.float64, torch.float64) else torch.float32
            out = torch.empty(self.shape, dtype=tdt, device=self.device)
            V.vsv_get_field(self.g, fid, out.data_ptr(), _dtype_code(tdt), 1)
            return out
        out = np.empty(self.shape, dtype=dtype)
        V.vsv_get_field(self.g, fid, out.ctypes.data, _dtype_code(dtype), 0)
        return out

    def set_field(self, fid, arr):
        if isinstance(arr, torch.Tensor):
            t = arr.contiguous()
            return V.vsv_set_field(self.g, fid, t.data_ptr(), _dtype_code(t.dtype), int(t.is_cuda))
        a = np.ascontiguousarray(arr)
        return V.vsv_set_field(self.g, fid, a.ctypes.data, _dtype_code(a.dtype.type), 0)

    def diagnostics(self):
        return V.vsv_get_diagnostics(self.g)

    def stress_profile(self):
        return V.vsv_get_stress_profile(self.g, self.ny)

    def solve_poisson(self, rhs, x0=None, periodic=(True, False, False), tol=1e-12,
                      max_cycles=200, check=True, shift=0.0):
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        x = np.zeros_like(rhs) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        st, cyc, rr = V.vsv_solve_poisson(self.g, rhs.ctypes.data, x.ctypes.data,
                                          V.VSV_DTYPE_F64, 0, periodic, tol, max_cycles,
                                          check=check, shift=shift)
        return x, cyc, rr, st

    def stability_limit(self):
        return V.vsv_stability_limit(self.g)

    def kernel_launches(self):
        return V.vsv_kernel_launches(self.g)

    def kernel_bytes(self):
        return V.vsv_kernel_bytes(self.g)

    def close(self):
        if self.g is not None:
            V.vsv_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent simulations stepped together through one captured CUDA
    graph (vsv_batch_*).  Give each simulation its own stream so that the
    small ones run concurrently; the batch orders itself after their queued
    work and they after it."""

    def __init__(self, sims, stream=None):
        self.sims = list(sims)
        dev = self.sims[0].device
        # a stream of its own: graphs cannot be captured on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        self.b = V.vsv_batch_create([s.g for s in self.sims], self.stream.cuda_stream)

    def step(self, nsteps, dt):
        return V.vsv_batch_step(self.b, nsteps, dt, grids=[s.g for s in self.sims])

    def close(self):
        if self.b is not None:
            V.vsv_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
