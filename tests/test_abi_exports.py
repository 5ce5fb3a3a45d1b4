"""The C-ABI library loads and exports every entry point include/cslbm.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

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


def _p3(n, lo, hi, tau=0.8, storage=None):
    return _abi.Params((ctypes.c_int * 3)(*n), (ctypes.c_int * 3)(*lo), (ctypes.c_int * 3)(*hi), tau, 0.0,
                       (ctypes.c_double * 3)(0, 0, 0), _abi.FP32 if storage is None else storage, 0)


def test_degenerate_and_maximum_sizes_without_gpu():
    """Sizes at the edges of what a context takes: an empty axis, a single
    node (periodic), a non-periodic axis of 2 nodes, the 32-bit field offsets
    (25 N < 2^32: the largest lattice is 171,798,691 nodes) and 65,535 planes."""
    lib = _abi.load()
    n = ctypes.c_size_t(0)
    P, W = 0, 1
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3((0, 4, 4), (P, P, P), (P, P, P))), ctypes.byref(n)) == _abi.EINVAL
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3((1, 1, 1), (P, P, P), (P, P, P))), ctypes.byref(n)) == _abi.OK
    assert n.value > 0
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3((4, 4, 2), (P, P, W), (P, P, W))), ctypes.byref(n)) == _abi.EINVAL
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3((4, 4, 3), (P, P, W), (P, P, W))), ctypes.byref(n)) == _abi.OK
    # 555 x 555 x 557 = 171,569,925 nodes (89 GB of FP32 workspace) fits; one more plane does not
    ok, big = (555, 555, 557), (555, 555, 558)
    assert 25 * np.prod(ok, dtype=np.int64) < 2 ** 32 <= 25 * np.prod(big, dtype=np.int64)
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3(ok, (P, P, W), (P, P, W))), ctypes.byref(n)) == _abi.OK
    per_node = n.value / np.prod(ok, dtype=np.int64)
    assert 300 < per_node < 1000 and n.value < 280e9  # fits the GPU's memory with room to spare
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3(big, (P, P, W), (P, P, W))), ctypes.byref(n)) == _abi.EINVAL
    assert b"too large" in lib.cslbm_last_error()
    assert lib.cslbm_workspace_bytes(ctypes.byref(_p3((4, 4, 65536), (P, P, P), (P, P, P))),
                                     ctypes.byref(n)) == _abi.EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises; there is no fallback."""
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi._build, "LIB", str(tmp_path / "libcslbm.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _abi.load(build_if_missing=False)
    monkeypatch.setattr(_abi._build, "nvcc", lambda: (_ for _ in ()).throw(RuntimeError("nvcc not found")))
    monkeypatch.setattr(_abi._build, "up_to_date", lambda: False)
    with pytest.raises(RuntimeError, match="nvcc"):
        _abi.load()


def test_create_validates_before_touching_the_device():
    """cslbm_create checks its arguments before any CUDA call: a null or
    misaligned workspace is EINVAL, a short one ENOMEM, and nothing is
    created (the pointer given is host memory and is never written)."""
    lib = _abi.load()
    p = _p3((16, 16, 8), (0, 0, 1), (0, 0, 1))
    need = ctypes.c_size_t(0)
    assert lib.cslbm_workspace_bytes(ctypes.byref(p), ctypes.byref(need)) == _abi.OK
    out = ctypes.c_void_p(0)
    buf = ctypes.create_string_buffer(1024 + 256)
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    assert lib.cslbm_create(ctypes.byref(p), None, need.value, None, ctypes.byref(out)) == _abi.EINVAL
    assert lib.cslbm_create(ctypes.byref(p), base + 8, need.value, None, ctypes.byref(out)) == _abi.EINVAL
    assert b"256-byte" in lib.cslbm_last_error()
    assert lib.cslbm_create(ctypes.byref(p), base, 1024, None, ctypes.byref(out)) == _abi.ENOMEM
    assert out.value is None
    p.tau = 0.4
    assert lib.cslbm_create(ctypes.byref(p), base, need.value, None, ctypes.byref(out)) == _abi.EINVAL
