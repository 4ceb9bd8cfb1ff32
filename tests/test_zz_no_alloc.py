"""The no-allocation volume/area entry point against the existing path.

Some callers of this library may not allocate device memory (a plugin
whose host application owns every device allocation, or a latency-critical
loop that cannot afford the synchronisation of cudaMalloc / cudaFree).
vsv_volume_area_static serves them with scratch in a fixed file-scope
device array.  This test calls it twice in a row through the C ABI, on two
different fields, and checks each result against the volume and area that
vsv_get_diagnostics reports for the same field.  Collected last on purpose.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-9   # relative, as for the other diagnostics parity checks


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


def _reference(V, w):
    from paper_2601_05031_gb300.sim import Simulation
    sim = Simulation.from_workload(w, V.VSV_FP64)
    sim.set_phi(w.phi0)
    d = sim.diagnostics()
    sim.close()
    return d["volume"], d["area"]


def _static(V, w):
    import torch
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = V.vsv_volume_area_static(phi.data_ptr(), w.nx, w.ny, w.nz, w.h, w.eps, w.z_periodic,
                                  out.data_ptr(), stream.cuda_stream)
    assert st == V.VSV_OK
    torch.cuda.synchronize()
    return float(out[0]), float(out[1])


def test_no_alloc_volume_area_two_calls_match_existing_path(V):
    w1 = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5)
    w2 = inputs.vesicle(32, 16, 16, inputs.COUETTE, 0.9, 1.5, b_range=(0.24, 0.28))
    for w in (w1, w2):      # two calls in a row share the static scratch
        v_ref, a_ref = _reference(V, w)
        v, a = _static(V, w)
        assert abs(v - v_ref) <= TOL * abs(v_ref), (v, v_ref)
        assert abs(a - a_ref) <= TOL * abs(a_ref), (a, a_ref)


def test_no_alloc_rejects_shapes_beyond_its_scratch(V):
    import torch
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = V.vsv_volume_area_static(dummy.data_ptr(), 2, 300, 300, 1.0, 1.0, 0, dummy.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert st == V.VSV_EINVAL


def test_no_alloc_rejects_host_memory(V):
    """phi and out must be device memory of the current device: a host
    buffer is refused before anything is launched (the kernels never see
    it), and a valid call afterwards still matches."""
    import torch
    host = torch.zeros(16 * 12 * 12, dtype=torch.float64)
    dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert V.vsv_volume_area_static(host.data_ptr(), 16, 12, 12, 1.0, 1.0, 0, dev.data_ptr(),
                                    stream) == V.VSV_EINVAL
    phi = torch.ones(16 * 12 * 12, dtype=torch.float64, device="cuda")
    assert V.vsv_volume_area_static(phi.data_ptr(), 16, 12, 12, 1.0, 1.0, 0, host.data_ptr(),
                                    stream) == V.VSV_EINVAL
    w = inputs.droplet_duct(nx=16, ny=12, nz=12, radius=3.5)
    v_ref, a_ref = _reference(V, w)
    v, a = _static(V, w)
    assert abs(v - v_ref) <= TOL * abs(v_ref) and abs(a - a_ref) <= TOL * abs(a_ref)
