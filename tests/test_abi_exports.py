"""The C-ABI library loads and exports every entry point include/cslbm.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_1803_07822_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:cslbm_status|const char\*)\s+(cslbm(?:2d)?_\w+)\s*\(", src, re.M))
    return names


def test_header_and_binding_agree():
    names = declared()
    assert len(names) >= 17
    assert names == set(_abi.SIGNATURES)


def test_library_exports_every_symbol():
    lib = _abi.load()
    for name in declared():
        assert hasattr(lib, name), name


def test_workspace_bytes_and_validation_without_gpu():
    lib = _abi.load()
    p = _abi.Params((ctypes.c_int * 3)(16, 16, 32), (ctypes.c_int * 3)(1, 0, 0), (ctypes.c_int * 3)(1, 0, 0),
                    0.8, 0.0, (ctypes.c_double * 3)(0, 0, 1e-4), _abi.FP32, 0)
    n = ctypes.c_size_t(0)
    assert lib.cslbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == _abi.OK
    N = 16 * 16 * 32
    assert n.value >= N * (2 * 19 * 4 + 2 * 10 * 4 + 2 * 25 * 4 + 9 * 8)
    p.tau = 0.5
    assert lib.cslbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == _abi.EINVAL
    assert b"tau" in lib.cslbm_last_error()
    p.tau = 0.8
    p.bc_hi[0] = 0  # periodic on one face only
    assert lib.cslbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == _abi.EINVAL


def test_2d_workspace_bytes_and_validation_without_gpu():
    lib = _abi.load()
    p = _abi.Params2D((ctypes.c_int * 2)(257, 65), (ctypes.c_int * 2)(2, 1), (ctypes.c_int * 2)(3, 1), 0.6, 0.0,
                      (ctypes.c_double * 2)(0, 0), _abi.FP32)
    n = ctypes.c_size_t(0)
    assert lib.cslbm2d_workspace_bytes(ctypes.byref(p), ctypes.byref(n)) == _abi.OK
    N = 257 * 65
    assert n.value >= N * (2 * 9 * 4 + 2 * 6 * 4 + 2 * 10 * 4 + 4 * 8)
    for bad in (dict(tau=0.4), dict(storage=_abi.FP16S)):
        q = _abi.Params2D((ctypes.c_int * 2)(257, 65), (ctypes.c_int * 2)(2, 1), (ctypes.c_int * 2)(3, 1),
                          bad.get("tau", 0.6), 0.0, (ctypes.c_double * 2)(0, 0), bad.get("storage", _abi.FP32))
        assert lib.cslbm2d_workspace_bytes(ctypes.byref(q), ctypes.byref(n)) == _abi.EINVAL
    q = _abi.Params2D((ctypes.c_int * 2)(257, 65), (ctypes.c_int * 2)(0, 1), (ctypes.c_int * 2)(3, 1), 0.6, 0.0,
                      (ctypes.c_double * 2)(0, 0), _abi.FP32)  # periodic on one side only
    assert lib.cslbm2d_workspace_bytes(ctypes.byref(q), ctypes.byref(n)) == _abi.EINVAL
