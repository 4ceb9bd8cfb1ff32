"""The C-ABI library loads, exports every function include/vsv.h declares,
and validates arguments on the host before touching a GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    from paper_2601_05031_gb300 import build
    build.build()
    from paper_2601_05031_gb300 import vsv
    return vsv


def _declared():
    txt = open(os.path.join(ROOT, "include", "vsv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vsv_[a-z_0-9]+)\s*\(", txt)))


def test_header_matches_binding(V):
    assert _declared() == sorted(V.EXPORTS)


def test_library_exports_every_declared_symbol(V):
    lib = V.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert V.vsv_version().startswith("vsv-gb300")


def test_workspace_bytes_host_only(V):
    n32 = V.vsv_workspace_bytes(48, 24, 24, V.VSV_MIXED)
    n64 = V.vsv_workspace_bytes(48, 24, 24, V.VSV_FP64)
    N = 48 * 24 * 24
    assert n32 > 13 * 4 * N and n64 > 13 * 8 * N
    assert V.vsv_workspace_bytes(0, 24, 24, V.VSV_MIXED) == 0
    assert V.vsv_workspace_bytes(8, 1, 8, V.VSV_MIXED) == 0
    assert V.vsv_workspace_bytes(8, 8, 8, 7) == 0


def test_create_rejects_bad_arguments_before_any_launch(V):
    lib = V.lib()
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)        # aligned, never dereferenced
    nb = V.vsv_workspace_bytes(16, 8, 8, V.VSV_MIXED)
    # odd periodic x
    assert lib.vsv_create(ctypes.byref(out), 15, 8, 8, 1.0, V.VSV_MIXED, fake, nb, None) == V.VSV_EINVAL
    # misaligned workspace
    assert lib.vsv_create(ctypes.byref(out), 16, 8, 8, 1.0, V.VSV_MIXED, ctypes.c_void_p(1 << 20 | 8),
                          nb, None) == V.VSV_EINVAL
    # too small
    assert lib.vsv_create(ctypes.byref(out), 16, 8, 8, 1.0, V.VSV_MIXED, fake, nb - 1, None) == V.VSV_ENOMEM
    # bad spacing / precision / null workspace
    assert lib.vsv_create(ctypes.byref(out), 16, 8, 8, 0.0, V.VSV_MIXED, fake, nb, None) == V.VSV_EINVAL
    assert lib.vsv_create(ctypes.byref(out), 16, 8, 8, 1.0, 5, fake, nb, None) == V.VSV_EINVAL
    assert lib.vsv_create(ctypes.byref(out), 16, 8, 8, 1.0, V.VSV_MIXED, None, nb, None) == V.VSV_EINVAL
    assert out.value is None


def test_null_handles_are_rejected(V):
    lib = V.lib()
    assert lib.vsv_step(None, 1, 0.1) == V.VSV_EINVAL
    assert lib.vsv_destroy(None) == V.VSV_OK
    assert lib.vsv_check(None) == V.VSV_EINVAL
    assert lib.vsv_state_bytes(None) == 0
    assert lib.vsv_kernel_launches(None) == 0
    assert lib.vsv_kernel_bytes(None) == 0.0
    assert lib.vsv_batch_step(None, 1, 0.1) == V.VSV_EINVAL
    assert lib.vsv_batch_destroy(None) == V.VSV_OK
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.vsv_batch_create(ctypes.byref(out), arr, 0, None) == V.VSV_EINVAL
    assert lib.vsv_batch_create(ctypes.byref(out), arr, 1, None) == V.VSV_EINVAL
    arr2 = (ctypes.c_void_p * 1)(1234)   # never dereferenced: the NULL stream is rejected first
    assert lib.vsv_batch_create(ctypes.byref(out), arr2, 1, None) == V.VSV_EINVAL
    assert out.value is None
    assert lib.vsv_tape_create(ctypes.byref(out), None, 20, 0.0) == V.VSV_EINVAL
    assert out.value is None
    assert lib.vsv_tape_destroy(None) == V.VSV_OK
    assert lib.vsv_tape_forward(None, None, V.VSV_DTYPE_F64, 1, 1, 0.1) == V.VSV_EINVAL
    assert lib.vsv_tape_backward(None, None, None, 1, None) == V.VSV_EINVAL
    assert lib.vsv_tape_bytes(None) == 0
    assert lib.vsv_tape_set_cycles(None, 3) == V.VSV_EINVAL
    assert lib.vsv_tape_info(None, None, None, None) == V.VSV_EINVAL
    p = V.vsv_default_solver(V.VSV_MIXED)
    assert p.kind == V.VSV_SOLVER_MG and p.nu1 >= 1 and p.max_cycles > 0


def test_binding_structs_match_header_sizes(V):
    # field counts of the C structs as declared in the header
    txt = open(os.path.join(ROOT, "include", "vsv.h")).read()
    for cname, pyt in (("vsv_flow_params", V.vsv_flow_params), ("vsv_fe_params", V.vsv_fe_params),
                       ("vsv_solver_params", V.vsv_solver_params), ("vsv_bc", V.vsv_bc)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", txt).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"\b([a-z_0-9]+)\s*(?:\[\d+\])?\s*[;,]", body)
        assert [n for n, _ in pyt._fields_] == names, cname


def test_solver_defaults_and_autotune_launch_shapes(V):
    """The library's size-based launch defaults (component streams and
    programmatic dependent launches: 2, by grid size; level-by-level lower
    cycle) are the autotuner's untuned shape, and every candidate shape is
    one the solver accepts (the cooperative lower cycle without the
    component streams), with both launch-overlap settings among them."""
    from paper_2601_05031_gb300 import autotune
    p = V.vsv_default_solver(V.VSV_MIXED)
    assert (p.component_streams, p.launch_overlap, p.lower_cycle) == (2, 2, 0)
    assert autotune.TunedSchedule(2, 2, 0.0, 0.0, []).shape == (2, 2, 0)
    shapes = autotune.DEFAULT_SHAPES
    assert len(set(shapes)) == len(shapes)
    for cs, ov, lc in shapes:
        assert cs in (0, 1) and ov in (0, 1) and lc in (0, 1)
        assert not (lc and cs)
    assert {ov for _, ov, _ in shapes} == {0, 1}
