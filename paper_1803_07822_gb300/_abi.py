"""ctypes binding of the C ABI in ``include/cslbm.h`` (argument marshalling only).

Every function keeps the C name; pointers are passed as integers (device
addresses from torch tensors, host addresses from numpy arrays).  Loading
fails loudly when the library has not been built: there is no other path.
"""
from __future__ import annotations

import ctypes
import os

from . import buildlib as _build

OK, EINVAL, ECUDA, ENOMEM, EUNSTABLE, ETIMEOUT, ESTATE = range(7)
FP32, FP16S, BF16S, FP64 = range(4)
STEP_AUTO, STEP_FLAT, STEP_ROWS = range(3)
PERIODIC, WALL, INFLOW, OUTFLOW = range(4)

_STATUS = {0: "OK", 1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "EUNSTABLE", 5: "ETIMEOUT", 6: "ESTATE"}


class CslbmError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__(f"{func}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double), ("fext", ctypes.c_double * 3),
                ("storage", ctypes.c_int), ("transform_flags", ctypes.c_int),
                ("step_kernel", ctypes.c_int)]


class Params2D(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 2), ("bc_lo", ctypes.c_int * 2), ("bc_hi", ctypes.c_int * 2),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double), ("fext", ctypes.c_double * 2),
                ("storage", ctypes.c_int)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_D = ctypes.POINTER(ctypes.c_double)

# name -> argtypes (all return cslbm_status except cslbm_last_error)
SIGNATURES = {
    "cslbm_workspace_bytes": [ctypes.POINTER(Params), ctypes.POINTER(_SZ)],
    "cslbm_create": [ctypes.POINTER(Params), _P, _SZ, _P, ctypes.POINTER(_P)],
    "cslbm_destroy": [_P],
    "cslbm_set_metric": [_P, _P, _P, _I],
    "cslbm_set_jacobian": [_P, _P, _I],
    "cslbm_update_metric": [_P, _P, _P, _P, _I],
    "cslbm_update_metric_mixed": [_P, _P, _P, _P],
    "cslbm_init_equilibrium": [_P, _P, _P, _I],
    "cslbm_set_boundary_velocity": [_P, _I, _I, _P, _I],
    "cslbm_step": [_P, _I],
    "cslbm_get_moments": [_P, _P, _P, _I, _I],
    "cslbm_total_mass": [_P, _D],
    "cslbm_total_mass_static": [_P, _D],
    "cslbm_wall_force": [_P, _I, _I, _D],
    "cslbm_test_withhold_publication": [_P, _I, ctypes.c_longlong],
    "cslbm_check": [_P],
    "cslbm_state_bytes": [_P, ctypes.POINTER(_SZ)],
    "cslbm_save_state": [_P, _P, _SZ, _I],
    "cslbm_load_state": [_P, _P, _SZ, _I],
    "cslbm_profile_enable": [_P, _I],
    "cslbm_profile_read": [_P, _D, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
    "cslbm_adjoint_workspace_bytes": [_P, ctypes.POINTER(_SZ)],
    "cslbm_adjoint_attach": [_P, _P, _SZ],
    "cslbm_adjoint_seed_wall_force": [_P, _I, _I, _D],
    "cslbm_step_backward": [_P],
    "cslbm_adjoint_init_backward": [_P],
    "cslbm_adjoint_metric_grad": [_P, _P, _P, _P, _P, _P],
    "cslbm_transform_interp_scratch_bytes": [_P, ctypes.POINTER(_SZ)],
    "cslbm_update_metric_interp": [_P, _P, _P, _P, _P, _P, _SZ],
    "cslbm_lattice_gradient_scratch_bytes": [_P, _I, _I, ctypes.POINTER(_SZ)],
    "cslbm_lattice_gradient": [_P, _P, _I, _I, _P, _P, _SZ],
    "cslbm_metric_lattice_scratch_bytes": [_P, _I, ctypes.POINTER(_SZ)],
    "cslbm_set_metric_lattice": [_P, _P, _I, _P, _SZ],
    "cslbm_update_metric_lattice": [_P, _P, _P, _I, _P, _SZ],
    "cslbm_batch_workspace_bytes": [_I, ctypes.POINTER(Params), ctypes.POINTER(_SZ)],
    "cslbm_batch_create": [_I, ctypes.POINTER(Params), _P, _SZ, _P, ctypes.POINTER(_P)],
    "cslbm_batch_context": [_P, _I, ctypes.POINTER(_P)],
    "cslbm_batch_step": [_P, _I],
    "cslbm_batch_tune": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)],
    "cslbm_batch_tune_results": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)],
    "cslbm_batch_check": [_P],
    "cslbm_batch_set_shape": [_P, ctypes.POINTER(_I)],
    "cslbm_batch_launches": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "cslbm_batch_destroy": [_P],
    "cslbm2d_workspace_bytes": [ctypes.POINTER(Params2D), ctypes.POINTER(_SZ)],
    "cslbm2d_create": [ctypes.POINTER(Params2D), _P, _SZ, _P, ctypes.POINTER(_P)],
    "cslbm2d_destroy": [_P],
    "cslbm2d_set_metric": [_P, _P, _P, _I],
    "cslbm2d_set_jacobian": [_P, _P, _I],
    "cslbm2d_update_metric": [_P, _P, _P, _P, _I],
    "cslbm2d_set_boundary_velocity": [_P, _I, _I, _P, _I],
    "cslbm2d_init_equilibrium": [_P, _P, _P, _I],
    "cslbm2d_step": [_P, _I],
    "cslbm2d_get_moments": [_P, _P, _P, _I, _I],
    "cslbm2d_total_mass": [_P, _D],
    "cslbm2d_wall_force": [_P, _I, _I, _D],
    "cslbm_last_error": [],
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcslbm.so (building it in-tree first if it is missing)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "cslbm_last_error" else ctypes.c_int
        _lib = lib
    return _lib


def call(name, *args):
    """Call a status-returning entry point; raise CslbmError on failure."""
    lib = load()
    st = getattr(lib, name)(*args)
    if st != OK:
        raise CslbmError(st, name, lib.cslbm_last_error().decode())
    return st
