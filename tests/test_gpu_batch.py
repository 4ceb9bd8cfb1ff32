"""Batched stepping (vsv_batch_*): one captured CUDA graph of six steps of
several independent grids gives the same bits as stepping each grid alone."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_05031_gb300 import build
    build.build()
    from paper_2601_05031_gb300 import vsv
    vsv.lib()
    return vsv


def _make(V, w, prec, cycles, own_stream):
    import torch
    from paper_2601_05031_gb300.sim import Simulation
    stream = torch.cuda.Stream() if own_stream else None
    sim = Simulation.from_workload(w, prec, stream=stream)
    sp = sim.solver_params()
    sp.fixed_cycles = cycles
    sp.tol = 1e-7 if prec == V.VSV_MIXED else 1e-12
    V.vsv_set_solver(sim.g, sp)
    sim.set_phi(w.phi0)
    return sim


def _state(V, sim):
    f = [sim.field(V.VSV_FIELD_PHI)]
    f += [sim.field(V.VSV_FIELD_OMEGA_PERT_X + c) for c in range(3)]
    f += [sim.field(V.VSV_FIELD_PSI_PERT_X + c) for c in range(3)]
    return f


@pytest.mark.parametrize("prec,nsteps", [("mixed", 15), ("fp64", 8)])
def test_batch_matches_individual_steps(V, prec, nsteps):
    from paper_2601_05031_gb300.sim import Batch
    P = V.VSV_MIXED if prec == "mixed" else V.VSV_FP64
    ws = inputs.batch_instances(n=3, seed=3, nsteps=nsteps)
    ws.append(inputs.vesicle_couette_512x256x256(nx=128, ny=32, nz=32))  # tile-aligned kernels
    ref = []
    for w in ws:
        sim = _make(V, w, P, 2, False)
        sim.step(nsteps, w.dt)
        ref.append(_state(V, sim))
        sim.close()
    sims = [_make(V, w, P, 2, True) for w in ws]
    b = Batch(sims)
    b.step(nsteps, ws[0].dt)
    for sim, r in zip(sims, ref):
        got = _state(V, sim)
        for a, c in zip(got, r):
            assert np.array_equal(a, c)
        d = sim.diagnostics()
        assert d["steps"] == nsteps
    # a second call replays the captured graph again
    b.step(6, ws[0].dt)
    assert all(s.diagnostics()["steps"] == nsteps + 6 for s in sims)
    b.close()
    for s in sims:
        s.close()


def test_batch_needs_fixed_cycles(V):
    from paper_2601_05031_gb300.sim import Batch
    w = inputs.batch_instances(n=1, seed=5)[0]
    sim = _make(V, w, V.VSV_MIXED, 0, True)
    b = Batch([sim])
    with pytest.raises(V.VsvError) as e:
        b.step(6, w.dt)
    assert e.value.status == V.VSV_EINVAL
    b.close()
    sim.close()


def test_autotune_picks_cheapest_schedule_meeting_target(V):
    from paper_2601_05031_gb300 import autotune
    w = inputs.vesicle(64, 32, 32, inputs.COUETTE, 0.9, 1.0, dt=1e-4, b_range=(0.2, 0.24))
    cands = ((1, 1), (2, 1), (4, 1), (6, 1))
    s = autotune.tune(w, target=1e-6, steps=4, candidates=cands, use_cache=False)
    ok = [t for t in s.trials if t["vel_err"] * 3.0 <= 1e-6]
    assert ok, s.trials
    assert s.vel_err * 3.0 <= 1e-6
    best = min(ok, key=lambda t: t["ms_per_step"])
    assert (s.fixed_cycles, s.extrapolate) == (best["fixed_cycles"], best["extrapolate"])
    # the tiling mode is the faster of the two timed on that schedule
    assert set(s.tiling_ms) == {0, 2} and s.tiling_ms[s.variant] == min(s.tiling_ms.values())
    # the launch shape is the fastest timed on that schedule and mode; the
    # cooperative lower cycle is a candidate on variant 0 only
    shapes = set(autotune.DEFAULT_SHAPES)
    if s.variant != 0:
        shapes = {t for t in shapes if not t[2]}
    assert set(s.shape_ms) == shapes
    assert s.ms_per_step == s.shape_ms[s.shape] == min(s.shape_ms.values())
    # applied to a simulation, the tuned schedule is what its solver runs
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, V.VSV_MIXED)
    autotune.apply(sim, s)
    sim.set_phi(w.phi0)
    sim.step(2, w.dt)
    assert V.vsv_check(sim.g, check=False) == V.VSV_OK
    sim.close()
    # errors shrink with more cycles
    errs = [t["vel_err"] for t in s.trials]
    assert errs[0] > errs[-1]
    # the cache serves the size class without re-running
    s1 = autotune.tune(w, steps=4, candidates=cands)
    s2 = autotune.tune(w, steps=4, candidates=cands)
    assert s1 is s2
