"""Thin Python binding of the C ABI in include/vsv.h (argument marshalling
only).  Every function keeps the C name; every step of the time integration
runs in the CUDA kernels of libvsv.so.  Torch is used for device memory and
streams only.  Importing this module loads the library and raises if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvsv.so")

# ---------------------------------------------------------------- enums
VSV_OK, VSV_EINVAL, VSV_ENOMEM, VSV_ECUDA, VSV_ENOCONV, VSV_ENONFINITE, VSV_EUNSTABLE, VSV_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
STATUS_NAMES = {0: "VSV_OK", -1: "VSV_EINVAL", -2: "VSV_ENOMEM", -3: "VSV_ECUDA",
                -4: "VSV_ENOCONV", -5: "VSV_ENONFINITE", -6: "VSV_EUNSTABLE", -7: "VSV_ESTATE"}
VSV_FP64, VSV_MIXED = 0, 1
VSV_POISEUILLE_DUCT, VSV_POISEUILLE_PLANAR, VSV_COUETTE, VSV_QUIESCENT = 0, 1, 2, 3
VSV_CAHN_HILLIARD, VSV_HELFRICH = 0, 1
VSV_SOLVER_MG, VSV_SOLVER_SOR = 0, 1
VSV_DTYPE_F32, VSV_DTYPE_F64 = 0, 1
VSV_HOST_ASYNC = 2   # on_device: page-locked host memory, asynchronous (see the header)
(VSV_FIELD_PHI, VSV_FIELD_MU, VSV_FIELD_OMEGA_X, VSV_FIELD_OMEGA_Y, VSV_FIELD_OMEGA_Z,
 VSV_FIELD_PSI_X, VSV_FIELD_PSI_Y, VSV_FIELD_PSI_Z, VSV_FIELD_VEL_X, VSV_FIELD_VEL_Y,
 VSV_FIELD_VEL_Z, VSV_FIELD_STRESS_T, VSV_FIELD_OMEGA_PERT_X, VSV_FIELD_OMEGA_PERT_Y,
 VSV_FIELD_OMEGA_PERT_Z, VSV_FIELD_PSI_PERT_X, VSV_FIELD_PSI_PERT_Y, VSV_FIELD_PSI_PERT_Z,
 VSV_FIELD_COUNT) = range(19)
(VSV_KCLASS_SMOOTH, VSV_KCLASS_SMOOTH_FINE, VSV_KCLASS_RESTRICT, VSV_KCLASS_PROLONG,
 VSV_KCLASS_PHASE, VSV_KCLASS_ADJOINT, VSV_KCLASS_COUNT) = range(7)


class vsv_flow_params(C.Structure):
    _fields_ = [("kind", C.c_int), ("u_max", C.c_double), ("v_lo", C.c_double),
                ("v_hi", C.c_double), ("eta", C.c_double), ("rho", C.c_double)]


class vsv_fe_params(C.Structure):
    _fields_ = [("kind", C.c_int), ("sigma", C.c_double), ("kappa", C.c_double),
                ("eps", C.c_double), ("mobility", C.c_double), ("k_area", C.c_double),
                ("k_vol", C.c_double), ("mu_prefactor_half", C.c_int)]


class vsv_wall_motion(C.Structure):
    _fields_ = [("ramp", C.c_double * 2), ("amplitude", C.c_double * 2),
                ("frequency", C.c_double * 2), ("phase", C.c_double * 2)]


class vsv_solver_params(C.Structure):
    _fields_ = [("kind", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("fixed_cycles", C.c_int), ("check_every", C.c_int), ("nu1", C.c_int),
                ("nu2", C.c_int), ("max_levels", C.c_int), ("coarse_sweeps", C.c_int),
                ("omega_sor", C.c_double), ("variant", C.c_int), ("extrapolate", C.c_int),
                ("fixed_cycles_psi", C.c_int), ("omega_mg", C.c_double),
                ("lower_cycle", C.c_int), ("component_streams", C.c_int),
                ("launch_overlap", C.c_int)]


class vsv_bc(C.Structure):
    _fields_ = [("periodic", C.c_int * 3), ("shift", C.c_double)]


class vsv_diag(C.Structure):
    _fields_ = [("time", C.c_double), ("steps", C.c_int64), ("volume", C.c_double),
                ("area", C.c_double), ("volume0", C.c_double), ("area0", C.c_double),
                ("reduced_volume", C.c_double), ("energy", C.c_double),
                ("lambda_v", C.c_double), ("gamma_a", C.c_double), ("com", C.c_double * 3),
                ("dissipation", C.c_double), ("dissipation0", C.c_double),
                ("resistance_rel", C.c_double), ("omega_dev2", C.c_double),
                ("psi_dev2", C.c_double), ("max_div_v", C.c_double),
                ("max_div_psi", C.c_double), ("max_sigma_t", C.c_double),
                ("last_cycles_omega", C.c_int), ("last_cycles_psi", C.c_int),
                ("last_relres_omega", C.c_double), ("last_relres_psi", C.c_double),
                ("nonfinite", C.c_int)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "com" else v
        return out


# exported names, in header order (used by the ABI test)
EXPORTS = [
    "vsv_version", "vsv_workspace_bytes", "vsv_create", "vsv_destroy", "vsv_set_flow",
    "vsv_set_free_energy", "vsv_set_wall_motion", "vsv_set_solver", "vsv_default_solver", "vsv_set_phi", "vsv_step",
    "vsv_stability_limit", "vsv_solve_poisson", "vsv_get_field", "vsv_set_field",
    "vsv_get_diagnostics", "vsv_get_stress_profile", "vsv_state_bytes", "vsv_get_state",
    "vsv_set_state", "vsv_volume_area_static", "vsv_check", "vsv_barrier_check", "vsv_copy_wait_check",
    "vsv_last_error",
    "vsv_kernel_launches",
    "vsv_kernel_bytes", "vsv_profile_enable", "vsv_profile_read", "vsv_batch_create",
    "vsv_batch_step", "vsv_batch_destroy", "vsv_tape_create", "vsv_tape_workspace_bytes", "vsv_tape_create_in", "vsv_tape_destroy",
    "vsv_tape_forward", "vsv_tape_backward", "vsv_tape_set_cycles", "vsv_tape_bytes",
    "vsv_tape_info",
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(
            f"libvsv.so not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(path)
    vp, sz, i32, i64, dbl = C.c_void_p, C.c_size_t, C.c_int, C.c_int64, C.c_double
    sig = {
        "vsv_version": (C.c_char_p, []),
        "vsv_workspace_bytes": (sz, [i32, i32, i32, i32]),
        "vsv_create": (i32, [C.POINTER(vp), i32, i32, i32, dbl, i32, vp, sz, vp]),
        "vsv_destroy": (i32, [vp]),
        "vsv_set_flow": (i32, [vp, C.POINTER(vsv_flow_params)]),
        "vsv_set_free_energy": (i32, [vp, C.POINTER(vsv_fe_params)]),
        "vsv_set_wall_motion": (i32, [vp, C.POINTER(vsv_wall_motion)]),
        "vsv_set_solver": (i32, [vp, C.POINTER(vsv_solver_params)]),
        "vsv_default_solver": (i32, [C.POINTER(vsv_solver_params), i32]),
        "vsv_set_phi": (i32, [vp, vp, i32, i32]),
        "vsv_step": (i32, [vp, i32, dbl]),
        "vsv_stability_limit": (i32, [vp, C.POINTER(dbl)]),
        "vsv_solve_poisson": (i32, [vp, vp, vp, i32, i32, C.POINTER(vsv_bc), dbl, i32,
                                    C.POINTER(i32), C.POINTER(dbl)]),
        "vsv_get_field": (i32, [vp, i32, vp, i32, i32]),
        "vsv_set_field": (i32, [vp, i32, vp, i32, i32]),
        "vsv_get_diagnostics": (i32, [vp, C.POINTER(vsv_diag)]),
        "vsv_get_stress_profile": (i32, [vp, vp]),
        "vsv_state_bytes": (sz, [vp]),
        "vsv_get_state": (i32, [vp, vp, sz]),
        "vsv_set_state": (i32, [vp, vp, sz]),
        "vsv_volume_area_static": (i32, [vp, i32, i32, i32, dbl, dbl, i32, vp, vp]),
        "vsv_check": (i32, [vp]),
        "vsv_barrier_check": (i32, [vp, i32, i32, i32, dbl]),
        "vsv_copy_wait_check": (i32, [vp, i32, dbl]),
        "vsv_last_error": (C.c_char_p, [vp]),
        "vsv_kernel_launches": (i64, [vp]),
        "vsv_kernel_bytes": (dbl, [vp]),
        "vsv_profile_enable": (i32, [vp, i32, i32]),
        "vsv_profile_read": (i32, [vp, i32, C.POINTER(dbl), C.POINTER(i64), C.POINTER(dbl)]),
        "vsv_batch_create": (i32, [C.POINTER(vp), C.POINTER(vp), i32, vp]),
        "vsv_batch_step": (i32, [vp, i32, dbl]),
        "vsv_batch_destroy": (i32, [vp]),
        "vsv_tape_create": (i32, [C.POINTER(vp), vp, i32, dbl]),
        "vsv_tape_workspace_bytes": (i32, [vp, i32, i32, C.POINTER(C.c_size_t)]),
        "vsv_tape_create_in": (i32, [C.POINTER(vp), vp, i32, i32, dbl, vp, C.c_size_t]),
        "vsv_tape_destroy": (i32, [vp]),
        "vsv_tape_forward": (i32, [vp, vp, i32, i32, i32, dbl]),
        "vsv_tape_backward": (i32, [vp, vp, vp, i32, C.POINTER(dbl)]),
        "vsv_tape_set_cycles": (i32, [vp, i32]),
        "vsv_tape_bytes": (sz, [vp]),
        "vsv_tape_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class VsvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(handle, status, what):
    if status != VSV_OK:
        msg = lib().vsv_last_error(handle).decode() if handle else ""
        raise VsvError(status, f"{what}: {msg}")
    return status


# ---------------------------------------------------------------- same-name wrappers
def vsv_version() -> str:
    return lib().vsv_version().decode()


def vsv_workspace_bytes(nx, ny, nz, precision) -> int:
    return lib().vsv_workspace_bytes(nx, ny, nz, precision)


def vsv_create(nx, ny, nz, h, precision, workspace_ptr, ws_bytes, stream_ptr):
    out = C.c_void_p()
    st = lib().vsv_create(C.byref(out), nx, ny, nz, h, precision, C.c_void_p(workspace_ptr),
                          ws_bytes, C.c_void_p(stream_ptr))
    if st != VSV_OK:
        raise VsvError(st, "vsv_create")
    return out


def vsv_destroy(g):
    return lib().vsv_destroy(g)


def vsv_set_flow(g, kind, u_max=0.0, v_lo=0.0, v_hi=0.0, eta=1.0, rho=0.0):
    p = vsv_flow_params(kind, u_max, v_lo, v_hi, eta, rho)
    return _check(g, lib().vsv_set_flow(g, C.byref(p)), "vsv_set_flow")


def vsv_set_free_energy(g, kind, sigma=1.0, kappa=0.0, eps=1.0, mobility=1.0, k_area=0.0,
                        k_vol=0.0, mu_prefactor_half=0):
    p = vsv_fe_params(kind, sigma, kappa, eps, mobility, k_area, k_vol, mu_prefactor_half)
    return _check(g, lib().vsv_set_free_energy(g, C.byref(p)), "vsv_set_free_energy")


def vsv_set_wall_motion(g, motion, check=True):
    """motion: None (steady walls) or (ramp, amplitude, frequency, phase),
    each a pair (wall 0, wall 1)."""
    if motion is None:
        st = lib().vsv_set_wall_motion(g, None)
    else:
        ramp, amp, freq, phase = motion
        m = vsv_wall_motion((C.c_double * 2)(*ramp), (C.c_double * 2)(*amp),
                            (C.c_double * 2)(*freq), (C.c_double * 2)(*phase))
        st = lib().vsv_set_wall_motion(g, C.byref(m))
    return _check(g, st, "vsv_set_wall_motion") if check else st


def vsv_default_solver(precision) -> vsv_solver_params:
    p = vsv_solver_params()
    lib().vsv_default_solver(C.byref(p), precision)
    return p


def vsv_set_solver(g, params: vsv_solver_params):
    return _check(g, lib().vsv_set_solver(g, C.byref(params)), "vsv_set_solver")


def vsv_set_phi(g, ptr, dtype, on_device, check=True):
    st = lib().vsv_set_phi(g, C.c_void_p(ptr), dtype, on_device)
    return _check(g, st, "vsv_set_phi") if check else st


def vsv_step(g, nsteps, dt, check=True):
    st = lib().vsv_step(g, nsteps, dt)
    return _check(g, st, "vsv_step") if check else st


def vsv_stability_limit(g) -> float:
    d = C.c_double()
    _check(g, lib().vsv_stability_limit(g, C.byref(d)), "vsv_stability_limit")
    return d.value


def vsv_solve_poisson(g, rhs_ptr, x_ptr, dtype, on_device, periodic, tol, max_cycles, check=True,
                      shift=0.0):
    bc = vsv_bc((C.c_int * 3)(*[int(bool(p)) for p in periodic]), shift)
    cyc, rr = C.c_int(), C.c_double()
    st = lib().vsv_solve_poisson(g, C.c_void_p(rhs_ptr), C.c_void_p(x_ptr), dtype, on_device,
                                 C.byref(bc), tol, max_cycles, C.byref(cyc), C.byref(rr))
    if check:
        _check(g, st, "vsv_solve_poisson")
    return st, cyc.value, rr.value


def vsv_get_field(g, field, ptr, dtype, on_device):
    return _check(g, lib().vsv_get_field(g, field, C.c_void_p(ptr), dtype, on_device),
                  "vsv_get_field")


def vsv_set_field(g, field, ptr, dtype, on_device):
    return _check(g, lib().vsv_set_field(g, field, C.c_void_p(ptr), dtype, on_device),
                  "vsv_set_field")


def vsv_get_diagnostics(g) -> dict:
    d = vsv_diag()
    _check(g, lib().vsv_get_diagnostics(g, C.byref(d)), "vsv_get_diagnostics")
    return d.as_dict()


def vsv_get_stress_profile(g, ny):
    import numpy as np
    out = np.zeros(ny, dtype=np.float64)
    _check(g, lib().vsv_get_stress_profile(g, out.ctypes.data), "vsv_get_stress_profile")
    return out


def vsv_state_bytes(g) -> int:
    return lib().vsv_state_bytes(g)


def vsv_get_state(g, ptr, nbytes):
    return _check(g, lib().vsv_get_state(g, C.c_void_p(ptr), nbytes), "vsv_get_state")


def vsv_set_state(g, ptr, nbytes):
    return _check(g, lib().vsv_set_state(g, C.c_void_p(ptr), nbytes), "vsv_set_state")


def vsv_volume_area_static(phi_ptr, nx, ny, nz, h, eps, z_periodic, out_ptr, stream_ptr):
    """Volume and area of an FP64 device field into out_ptr (2 device
    doubles) with no device allocation; returns the vsv_status."""
    return lib().vsv_volume_area_static(C.c_void_p(phi_ptr), nx, ny, nz, h, eps, int(z_periodic),
                                        C.c_void_p(out_ptr), C.c_void_p(stream_ptr))


def vsv_check(g, check=True):
    st = lib().vsv_check(g)
    return _check(g, st, "vsv_check") if check else st


def vsv_barrier_check(g, blocks, rounds, extra_arrivals, limit_ms):
    """Bounded grid barrier check (see the header); returns the vsv_status."""
    return lib().vsv_barrier_check(g, blocks, rounds, extra_arrivals, limit_ms)


def vsv_copy_wait_check(g, probe_bytes, limit_ms):
    """Bounded copy-wait check of the fused sweep (see the header); returns
    the vsv_status."""
    return lib().vsv_copy_wait_check(g, probe_bytes, limit_ms)


def vsv_last_error(g) -> str:
    return lib().vsv_last_error(g).decode()


def vsv_kernel_launches(g) -> int:
    return lib().vsv_kernel_launches(g)


def vsv_kernel_bytes(g) -> float:
    return lib().vsv_kernel_bytes(g)


def vsv_profile_enable(g, kclass, enable=True):
    return _check(g, lib().vsv_profile_enable(g, kclass, int(enable)), "vsv_profile_enable")


def vsv_profile_read(g, kclass, with_bytes=False):
    """(total_ms, launches), or (total_ms, launches, algorithmic_bytes)."""
    ms, n, b = C.c_double(), C.c_int64(), C.c_double()
    _check(g, lib().vsv_profile_read(g, kclass, C.byref(ms), C.byref(n), C.byref(b)),
           "vsv_profile_read")
    return (ms.value, n.value, b.value) if with_bytes else (ms.value, n.value)


def vsv_batch_create(grids, stream_ptr):
    """grids: vsv_grid handles (c_void_p); returns the batch handle."""
    arr = (C.c_void_p * len(grids))(*[g.value if isinstance(g, C.c_void_p) else g for g in grids])
    out = C.c_void_p()
    st = lib().vsv_batch_create(C.byref(out), arr, len(grids), C.c_void_p(stream_ptr))
    if st != VSV_OK:
        raise VsvError(st, "vsv_batch_create")
    return out


def vsv_batch_step(b, nsteps, dt, grids=()):
    st = lib().vsv_batch_step(b, nsteps, dt)
    if st != VSV_OK:
        msg = "; ".join(lib().vsv_last_error(g).decode() for g in grids)
        raise VsvError(st, f"vsv_batch_step: {msg}")
    return st


def vsv_batch_destroy(b):
    return lib().vsv_batch_destroy(b)


def vsv_tape_create(g, every, tol=0.0):
    out = C.c_void_p()
    st = lib().vsv_tape_create(C.byref(out), g, every, tol)
    if st != VSV_OK:
        _check(g, st, "vsv_tape_create")
    return out


def vsv_tape_workspace_bytes(g, every, max_steps):
    """Device bytes of a tape over caller-owned memory (see the header)."""
    n = C.c_size_t()
    _check(g, lib().vsv_tape_workspace_bytes(g, every, max_steps, C.byref(n)),
           "vsv_tape_workspace_bytes")
    return n.value


def vsv_tape_create_in(g, every, max_steps, tol, workspace_ptr, workspace_bytes, check=True):
    """A tape whose device memory is the caller's workspace (see the
    header); returns the handle, or (handle, status) with check=False."""
    out = C.c_void_p()
    st = lib().vsv_tape_create_in(C.byref(out), g, every, max_steps, tol,
                                  C.c_void_p(workspace_ptr), workspace_bytes)
    if not check:
        return out, st
    if st != VSV_OK:
        _check(g, st, "vsv_tape_create_in")
    return out


def vsv_tape_destroy(t):
    return lib().vsv_tape_destroy(t)


def vsv_tape_forward(t, g, phi0_ptr, dtype, on_device, nsteps, dt):
    return _check(g, lib().vsv_tape_forward(t, C.c_void_p(phi0_ptr), dtype, int(on_device),
                                            nsteps, dt), "vsv_tape_forward")


def vsv_tape_backward(t, g, phibar_ptr, phibar0_ptr, on_device):
    """Returns (dJ/dkappa, dJ/dsigma); dJ/dphi^0 is written to phibar0_ptr."""
    pb = (C.c_double * 2)()
    _check(g, lib().vsv_tape_backward(t, C.c_void_p(phibar_ptr), C.c_void_p(phibar0_ptr),
                                      int(on_device), pb), "vsv_tape_backward")
    return pb[0], pb[1]


def vsv_tape_set_cycles(t, g, fixed_cycles):
    return _check(g, lib().vsv_tape_set_cycles(t, fixed_cycles), "vsv_tape_set_cycles")


def vsv_tape_bytes(t) -> int:
    return lib().vsv_tape_bytes(t)


def vsv_tape_info(t):
    """(adjoint solve cycles, re-run steps, checkpoints) of the last backward pass."""
    a, r, c = C.c_int64(), C.c_int64(), C.c_int()
    lib().vsv_tape_info(t, C.byref(a), C.byref(r), C.byref(c))
    return a.value, r.value, c.value
