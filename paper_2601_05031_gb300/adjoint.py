"""Gradients of a trajectory through the library's discrete adjoint.

``Tape`` wraps the C tape (vsv_tape_*): a checkpointed forward run from phi^0
and the reverse pass that returns dJ/dphi^0, dJ/dkappa and dJ/dsigma for a
given dJ/dphi^N.  ``trajectory`` exposes the map (phi^0, kappa, sigma) ->
phi^N as a torch.autograd.Function, so a loss written in torch on phi^N
back-propagates through the hand-written adjoint kernels.  This module only
marshals arguments; every step, forward and reverse, runs in libvsv.so.
"""
from __future__ import annotations

import torch

from . import vsv as V
from .sim import Simulation


class Tape:
    """A trajectory tape bound to a configured Simulation.

    ``every``: steps between checkpoints; ``tol``: relative residual of the
    adjoint Poisson solves (0: the library's default 1e-11).  The tape's
    device memory (segment record, adjoint fields, checkpoints) is a torch
    tensor owned here and handed to the library (vsv_tape_create_in); it is
    sized at the first forward pass and grown when a longer one comes."""

    def __init__(self, sim: Simulation, fe: dict, every: int = 20, tol: float = 0.0):
        self.sim = sim
        self.fe = dict(fe)
        self.every = every
        self.tol = tol
        self.t = None
        self.ws = None
        self.max_steps = 0
        self.fixed = 0

    def _bind(self, nsteps: int):
        """The C tape over a workspace for forward passes of nsteps steps."""
        if self.t is not None and nsteps <= self.max_steps:
            return
        if self.t is not None:
            V.vsv_tape_destroy(self.t)
            self.t = None
        nbytes = V.vsv_tape_workspace_bytes(self.sim.g, self.every, nsteps)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.sim.device)
        self.t = V.vsv_tape_create_in(self.sim.g, self.every, nsteps, self.tol,
                                      self.ws.data_ptr(), nbytes)
        self.max_steps = nsteps
        if self.fixed:
            V.vsv_tape_set_cycles(self.t, self.sim.g, self.fixed)

    @classmethod
    def from_workload(cls, w, precision=V.VSV_MIXED, every=20, tol=0.0, solver=None, stream=None):
        sim = Simulation.from_workload(w, precision, solver=solver, stream=stream)
        fe = dict(kind=w.fe_kind, sigma=w.sigma, kappa=w.kappa, eps=w.eps, mobility=w.mobility,
                  k_area=w.k_area, k_vol=w.k_vol)
        return cls(sim, fe, every, tol)

    def set_cycles(self, fixed_cycles: int):
        """Fixed cycles per adjoint solve (no host synchronisation); 0 solves
        to the tape's tolerance."""
        self.fixed = int(fixed_cycles)
        if self.t is not None:
            V.vsv_tape_set_cycles(self.t, self.sim.g, self.fixed)

    def set_params(self, kappa: float, sigma: float):
        self.fe["kappa"], self.fe["sigma"] = float(kappa), float(sigma)
        f = self.fe
        V.vsv_set_free_energy(self.sim.g, f["kind"], f["sigma"], f["kappa"], f["eps"],
                              f["mobility"], f["k_area"], f["k_vol"])

    def forward(self, phi0: torch.Tensor, nsteps: int, dt: float) -> torch.Tensor:
        """phi^N (FP64 device tensor) after nsteps steps from phi0."""
        p0 = phi0.detach().to(device=self.sim.device, dtype=torch.float64).contiguous()
        self._bind(nsteps)
        V.vsv_tape_forward(self.t, self.sim.g, p0.data_ptr(), V.VSV_DTYPE_F64, 1, nsteps, dt)
        return self.sim.field(V.VSV_FIELD_PHI, torch.float64, on_device=True)

    def backward(self, phibar: torch.Tensor):
        """(dJ/dphi^0 tensor, dJ/dkappa, dJ/dsigma) for phibar = dJ/dphi^N."""
        if self.t is None:
            raise RuntimeError("Tape.backward needs a forward pass first")
        pb = phibar.detach().to(device=self.sim.device, dtype=torch.float64).contiguous()
        out = torch.empty_like(pb)
        dk, ds = V.vsv_tape_backward(self.t, self.sim.g, pb.data_ptr(), out.data_ptr(), 1)
        return out, dk, ds

    def info(self):
        if self.t is None:
            return {"adjoint_cycles": 0, "recomputed_steps": 0, "checkpoints": 0, "device_bytes": 0}
        cyc, rerun, nck = V.vsv_tape_info(self.t)
        return {"adjoint_cycles": cyc, "recomputed_steps": rerun, "checkpoints": nck,
                "device_bytes": V.vsv_tape_bytes(self.t)}

    def close(self):
        if self.t is not None:
            V.vsv_tape_destroy(self.t)
            self.t = None
        self.ws = None
        if self.sim is not None:
            self.sim.close()
            self.sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, kappa, sigma, tape, nsteps, dt):
        tape.set_params(float(kappa), float(sigma))
        ctx.tape = tape
        return tape.forward(phi0, nsteps, dt)

    @staticmethod
    def backward(ctx, grad_phi):
        pb0, dk, ds = ctx.tape.backward(grad_phi)
        dev = grad_phi.device
        return (pb0, torch.tensor(dk, dtype=torch.float64, device=dev),
                torch.tensor(ds, dtype=torch.float64, device=dev), None, None, None)


def trajectory(phi0: torch.Tensor, kappa: torch.Tensor, sigma: torch.Tensor, tape: Tape,
               nsteps: int, dt: float) -> torch.Tensor:
    """phi^N of nsteps steps from phi0 with bending modulus kappa and
    tension sigma (0-dim tensors), differentiable in all three."""
    return _Trajectory.apply(phi0, kappa, sigma, tape, nsteps, dt)
