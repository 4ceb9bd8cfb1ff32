"""The Couette workload at its full size, 512 x 256 x 256, over 500 steps
(vesicle of reduced volume 0.9, kappa = 1, walls at +-0.05, eps = 1.5),
mixed path in the schedule bench.py times: the wall-normal profile of the
mean shear stress <sigma_xy>(y), the hydrodynamic resistance (dissipation
relative to the body-free flow) and the shape diagnostics, against the
plain FP64 path run with the same schedule."""
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


def test_500_steps_stress_profile_and_resistance(V):
    import torch
    import bench
    w = inputs.vesicle_couette_512x256x256()
    out = {}
    for name, prec in (("mixed", V.VSV_MIXED), ("fp64", V.VSV_FP64)):
        sim = bench.make_sim(w, prec, 4, 1)
        sim.step(w.nsteps, w.dt)
        d = sim.diagnostics()
        out[name] = {"diag": d, "profile": sim.stress_profile(),
                     "phi": sim.field(V.VSV_FIELD_PHI, np.float64, on_device=True).cpu(),
                     "vel": torch.stack([sim.field(V.VSV_FIELD_VEL_X + c, np.float64,
                                                   on_device=True).cpu() for c in range(3)])}
        sim.close()
        torch.cuda.empty_cache()
    m, f = out["mixed"], out["fp64"]
    prof_rel = float(np.linalg.norm(m["profile"] - f["profile"]) / np.linalg.norm(f["profile"]))
    res_rel = abs(m["diag"]["resistance_rel"] - f["diag"]["resistance_rel"]) / \
        abs(f["diag"]["resistance_rel"])
    phi_rel = float(torch.linalg.vector_norm(m["phi"] - f["phi"]) / torch.linalg.vector_norm(f["phi"]))
    vel_rel = float(torch.linalg.vector_norm(m["vel"] - f["vel"]) / torch.linalg.vector_norm(f["vel"]))
    keys = ("time", "reduced_volume", "energy", "dissipation", "dissipation0", "resistance_rel",
            "max_div_v")
    print("Couette 512x256x256, 500 steps:",
          {k: (m["diag"][k], f["diag"][k]) for k in keys})
    print("stress profile mixed vs FP64 %.3e, resistance %.3e, phi %.3e, velocity %.3e" %
          (prof_rel, res_rel, phi_rel, vel_rel))
    ny = w.ny
    print("<sigma_xy>(y) at y = 0, ny/4, ny/2, 3ny/4, ny-1:",
          [float(m["profile"][j]) for j in (0, ny // 4, ny // 2, 3 * ny // 4, ny - 1)])
    assert np.all(np.isfinite(m["profile"])) and np.isfinite(m["diag"]["resistance_rel"])
    # both paths take the same 4 V-cycles per solve; they differ by the FP32
    # arithmetic of the mixed path only
    assert phi_rel <= 1e-6 and vel_rel <= 1e-5, (phi_rel, vel_rel)
    assert prof_rel <= 1e-4 and res_rel <= 1e-4, (prof_rel, res_rel)
    # the body raises the dissipation above that of the plain Couette flow
    assert m["diag"]["resistance_rel"] > 0
