"""Fit membrane parameters to a target shape through the discrete adjoint.

The differentiable run: a Helfrich vesicle in duct Poiseuille flow (128 x 64
x 64 cells, x the flow axis), N forward steps from phi^0 with a checkpoint
every k steps.  A target phi* is made by the forward model itself at
(kappa*, sigma*); the loss is J = h^3/2 sum (phi^N - phi*)^2.  The run

1. takes the gradient of J in (phi^0, kappa, sigma) at the starting
   parameters through ``adjoint.trajectory`` (forward tape + reverse pass),
2. checks it against central differences of the forward map with step
   ``fd_step`` in kappa, sigma and a seeded smooth shape perturbation of
   phi^0 (``shape_direction``),
3. fits (kappa, sigma) with Adam (cosine-annealed step size), the gradient
   of every iteration coming from the adjoint, and prints one JSON line with the timings, the
   finite-difference agreement and the fit history.

    python -m paper_2601_05031_gb300.fit [--steps 200] [--every 20] [--adam 50]

Everything on the path runs in libvsv.so; this file marshals arguments and
runs the optimiser.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

import inputs
from . import vsv as V
from .adjoint import Tape, trajectory


def shape_direction(phi0: np.ndarray, seed: int) -> torch.Tensor:
    """A seeded perturbation of the body's shape: (1 - phi0^2) times a
    smooth field (a few low Fourier modes with normal coefficients), scaled
    to max-norm 1.  1 - phi^2 is the profile of d phi / dn, so adding it
    moves the interface along its normal by a smooth amount."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = phi0.shape
    z, y, x = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                          indexing="ij")
    s = np.zeros_like(phi0)
    for kx in range(3):
        for ky in range(3):
            for kz in range(3):
                c, ph = rng.standard_normal(), rng.uniform(0, 2 * np.pi)
                s += c * np.cos(2 * np.pi * kx * x + ph) * np.cos(np.pi * ky * y) * np.cos(np.pi * kz * z)
    d = (1.0 - phi0 ** 2) * s
    return torch.from_numpy(d / np.max(np.abs(d)))


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def run(nx=128, ny=64, nz=64, nsteps=200, every=20, kappa_true=2.0, sigma_true=0.5, kappa0=1.0,
        sigma0=0.0, adam_steps=50, lr=0.08, fd_step=1e-4, precision=V.VSV_MIXED, seed=0,
        solve_tol=None, adjoint_cycles=4):
    w = inputs.vesicle_poiseuille_128x64x64(seed=seed, nx=nx, ny=ny, nz=nz, nsteps=nsteps)
    dt = w.dt
    tape = Tape.from_workload(w, precision, every=every)
    sp = tape.sim.solver_params()
    if solve_tol is not None:
        sp.tol = solve_tol
    V.vsv_set_solver(tape.sim.g, sp)
    if adjoint_cycles:
        tape.set_cycles(adjoint_cycles)
    dev = tape.sim.device
    phi0 = torch.from_numpy(w.phi0).to(dev)
    h3 = w.h ** 3

    # target shape from the forward model at (kappa*, sigma*)
    tape.set_params(kappa_true, sigma_true)
    target = tape.forward(phi0, nsteps, dt).clone()

    def loss_of(phiN):
        return 0.5 * h3 * torch.sum((phiN - target) ** 2)

    def forward_loss(kappa, sigma, p0=phi0):
        tape.set_params(kappa, sigma)
        return float(loss_of(tape.forward(p0, nsteps, dt)))

    # 1. gradient at the starting point
    p0 = phi0.clone().requires_grad_(True)
    kap = torch.tensor(kappa0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sigma0, dtype=torch.float64, requires_grad=True)
    phiN, t_fwd = _timed(lambda: trajectory(p0, kap, sig, tape, nsteps, dt))
    J0 = loss_of(phiN)
    # time the adjoint stencil kernels of this backward pass by CUDA events
    V.vsv_profile_enable(tape.sim.g, V.VSV_KCLASS_ADJOINT, True)
    _, t_bwd = _timed(lambda: J0.backward())
    adj_ms, adj_launches, adj_bytes = V.vsv_profile_read(tape.sim.g, V.VSV_KCLASS_ADJOINT,
                                                         with_bytes=True)
    V.vsv_profile_enable(tape.sim.g, V.VSV_KCLASS_ADJOINT, False)
    info = tape.info()
    g_kappa, g_sigma = float(kap.grad), float(sig.grad)
    g_phi0 = p0.grad.detach()

    # 2. central differences of the forward map
    fd = {}
    for name, base, grad in (("kappa", kappa0, g_kappa), ("sigma", sigma0, g_sigma)):
        args_p = (base + fd_step, sigma0) if name == "kappa" else (kappa0, base + fd_step)
        args_m = (base - fd_step, sigma0) if name == "kappa" else (kappa0, base - fd_step)
        d = (forward_loss(*args_p) - forward_loss(*args_m)) / (2 * fd_step)
        fd[name] = {"fd": d, "adjoint": grad, "rel_err": abs(d - grad) / abs(d)}
    direction = shape_direction(w.phi0, seed + 1).to(dev)
    d = (forward_loss(kappa0, sigma0, phi0 + fd_step * direction) -
         forward_loss(kappa0, sigma0, phi0 - fd_step * direction)) / (2 * fd_step)
    ad = float(torch.sum(g_phi0 * direction))
    fd["phi0_direction"] = {"fd": d, "adjoint": ad, "rel_err": abs(d - ad) / abs(d)}

    # 3. Adam on (kappa, sigma); kappa kept positive (projected step)
    kap = torch.tensor(kappa0, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sigma0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([kap, sig], lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=max(1, adam_steps))
    hist = []
    t_fit0 = time.perf_counter()
    for it in range(adam_steps):
        opt.zero_grad()
        J = loss_of(trajectory(phi0, kap, sig, tape, nsteps, dt))
        J.backward()
        hist.append({"iter": it, "loss": float(J), "kappa": float(kap), "sigma": float(sig)})
        opt.step()
        sched.step()
        with torch.no_grad():
            kap.clamp_(min=0.05)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t_fit0
    J_end = forward_loss(float(kap), float(sig))
    ncell = w.nx * w.ny * w.nz
    out = {
        "workload": w.name, "precision": "mixed" if precision == V.VSV_MIXED else "fp64",
        "steps": nsteps, "checkpoint_every": every, "dt": dt,
        "adjoint_solves": (f"{adjoint_cycles} fixed cycles" if adjoint_cycles
                           else "to a relative residual of 1e-11"),
        "target": {"kappa": kappa_true, "sigma": sigma_true},
        "start": {"kappa": kappa0, "sigma": sigma0, "loss": float(J0)},
        "gradient": {"kappa": g_kappa, "sigma": g_sigma,
                     "phi0_norm": float(torch.linalg.vector_norm(g_phi0))},
        "timing_s": {"forward_tape": t_fwd, "backward": t_bwd,
                     "adam_total": t_fit, "adam_per_iter": t_fit / max(1, adam_steps)},
        "throughput_mcell_steps_s": {
            "forward_tape": ncell * nsteps / t_fwd / 1e6,
            "backward": ncell * nsteps / t_bwd / 1e6},
        "tape": info,
        "adjoint_kernels": {"ms": adj_ms, "launches": adj_launches, "alg_bytes": adj_bytes,
                            "share_of_backward": adj_ms / 1e3 / t_bwd,
                            "achieved_gbs": adj_bytes / (adj_ms / 1e3) / 1e9 if adj_ms > 0 else None},
        "finite_differences": {"step": fd_step, **fd},
        "fit": {"final": {"kappa": float(kap), "sigma": float(sig), "loss": J_end},
                "loss_ratio": J_end / float(J0), "history": hist},
    }
    tape.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--adam", type=int, default=50)
    ap.add_argument("--lr", type=float, default=0.08)
    ap.add_argument("--fd-step", type=float, default=1e-4)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--adjoint-cycles", type=int, default=4,
                    help="fixed cycles per adjoint solve (0: to a relative residual of 1e-11)")
    ap.add_argument("--grid", type=int, nargs=3, default=(128, 64, 64), metavar=("NX", "NY", "NZ"))
    ap.add_argument("--out", default=None, help="also write the JSON here")
    a = ap.parse_args(argv)
    res = run(nx=a.grid[0], ny=a.grid[1], nz=a.grid[2], nsteps=a.steps, every=a.every,
              adam_steps=a.adam, lr=a.lr, fd_step=a.fd_step, adjoint_cycles=a.adjoint_cycles,
              precision=V.VSV_MIXED if a.precision == "mixed" else V.VSV_FP64)
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
