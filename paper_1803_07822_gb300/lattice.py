"""Python front end of the C ABI: one curved-space D3Q19 channel per object.

PyTorch supplies the device memory (the workspace is a uint8 tensor) and the
stream; every step of the method runs in the library's CUDA kernels.  Inputs
may be CUDA tensors (passed as device pointers) or numpy arrays (host
pointers; the library stages the copies).  There is no CPU path: without a
CUDA device the constructor raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import call

STORAGE = {"fp32": _abi.FP32, "fp16": _abi.FP16S, "bf16": _abi.BF16S, "fp64": _abi.FP64}
STEP_KERNEL = {"auto": _abi.STEP_AUTO, "flat": _abi.STEP_FLAT, "rows": _abi.STEP_ROWS}


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("cslbm needs a CUDA device (GB300); no CPU fallback exists")
    return torch


class CurvedLattice:
    """A D3Q19 lattice of shape n = (n0, n1, n2) carrying a metric field.

    bc_lo / bc_hi: per-axis face rules (PERIODIC, WALL, INFLOW, OUTFLOW);
    tau: BGK relaxation time; fext: contravariant body-force density;
    storage: "fp32", "fp16", "bf16" (weight-shifted, FP32 arithmetic) or
    "fp64"; literal_a2: transform a_(2) itself on chart changes;
    step_kernel: "auto" (fused row pass, else row pass, else flat pass),
    "rows" (row pass with a separate momentum kernel) or "flat".
    """

    def __init__(self, n, bc_lo=(0, 0, 0), bc_hi=None, tau=0.8, theta=0.0, fext=(0.0, 0.0, 0.0),
                 storage="fp32", literal_a2=False, step_kernel="auto", device=None, stream=None):
        torch = _torch()
        _abi.load()
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        bc_hi = bc_lo if bc_hi is None else bc_hi
        self.params = _abi.Params((ctypes.c_int * 3)(*self.n), (ctypes.c_int * 3)(*bc_lo),
                                  (ctypes.c_int * 3)(*bc_hi), float(tau), float(theta),
                                  (ctypes.c_double * 3)(*fext), STORAGE[storage], int(bool(literal_a2)),
                                  STEP_KERNEL[step_kernel])
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        nbytes = ctypes.c_size_t(0)
        call("cslbm_workspace_bytes", ctypes.byref(self.params), ctypes.byref(nbytes))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.ctx = ctypes.c_void_p()
        call("cslbm_create", ctypes.byref(self.params), self.workspace.data_ptr(), nbytes.value,
             self.stream.cuda_stream, ctypes.byref(self.ctx))

    # -- marshalling --------------------------------------------------------
    def _arg(self, a, rows):
        """(pointer, on_device, keep-alive) for an FP64 [rows, N]-shaped input."""
        if a is None:
            return None, 1, None
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.device.type != "cuda":
                a = a.detach().to(torch.float64).contiguous().numpy()
            else:
                t = a.detach().to(self.device, torch.float64).contiguous()
                if t.numel() != rows:
                    raise ValueError(f"expected {rows} values, got {t.numel()}")
                t.record_stream(self.stream)  # a converted copy may be read after this call returns
                return t.data_ptr(), 1, t
        h = np.ascontiguousarray(a, dtype=np.float64)
        if h.size != rows:
            raise ValueError(f"expected {rows} values, got {h.size}")
        return h.ctypes.data, 0, h

    def face_nodes(self, axis):
        return self.n[(axis + 1) % 3] * self.n[(axis + 2) % 3]

    # -- geometry -----------------------------------------------------------
    def set_metric(self, g6, dg18):
        p1, d1, k1 = self._arg(g6, 6 * self.N)
        p2, d2, k2 = self._arg(dg18, 18 * self.N)
        if d1 != d2:
            raise ValueError("g6 and dg18 must both be host or both device arrays")
        call("cslbm_set_metric", self.ctx, p1, p2, d1)

    def set_jacobian(self, J9):
        p, d, k = self._arg(J9, 9 * self.N)
        call("cslbm_set_jacobian", self.ctx, p, d)

    def update_metric(self, g6, dg18, J9):
        p1, d1, k1 = self._arg(g6, 6 * self.N)
        p2, d2, k2 = self._arg(dg18, 18 * self.N)
        p3, d3, k3 = self._arg(J9, 9 * self.N)
        if not (d1 == d2 == d3):
            raise ValueError("metric inputs must all be host or all device arrays")
        call("cslbm_update_metric", self.ctx, p1, p2, p3, d1)

    def update_metric_mixed(self, g6, dg18, J9):
        """update_metric with the derivatives and the Jacobian as FP32 CUDA
        tensors (the metric stays FP64): the same state for FP32-arithmetic
        storage, 156 instead of 264 bytes per node to upload."""
        torch = _torch()
        g = g6.detach().to(self.device, torch.float64).contiguous()
        d = dg18.detach().to(self.device, torch.float32).contiguous()
        J = J9.detach().to(self.device, torch.float32).contiguous()
        for t, rows in ((g, 6), (d, 18), (J, 9)):
            if t.numel() != rows * self.N:
                raise ValueError(f"expected {rows * self.N} values, got {t.numel()}")
        call("cslbm_update_metric_mixed", self.ctx, g.data_ptr(), d.data_ptr(), J.data_ptr())
        self._hold(g, d, J)

    def update_metric_interp(self, g6, dg18, J9, psi3):
        """Chart change with interpolation: every new node takes the old
        state's moments at psi3 [3, N] (old lattice coordinates of its point)."""
        torch = _torch()
        g = self._dev64(g6, 6)
        d = self._dev64(dg18, 18)
        J = self._dev64(J9, 9)
        ps = self._dev64(psi3, 3)
        nb = ctypes.c_size_t(0)
        call("cslbm_transform_interp_scratch_bytes", self.ctx, ctypes.byref(nb))
        scratch = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        call("cslbm_update_metric_interp", self.ctx, g.data_ptr(), d.data_ptr(), J.data_ptr(), ps.data_ptr(),
             scratch.data_ptr(), scratch.numel())
        self._hold(g, d, J, ps, scratch)

    def _hold(self, *tensors):
        """Device buffers an asynchronous call reads: marked as used on the
        context's stream, so that the allocator does not hand their memory out
        again before that stream has run the call."""
        for t in tensors:
            t.record_stream(self.stream)

    # -- lattice derivatives (App. D) ----------------------------------------
    def _dev64(self, a, rows):
        torch = _torch()
        t = torch.as_tensor(a, dtype=torch.float64, device=self.device).reshape(rows, self.N).contiguous()
        return t

    def lattice_gradient(self, f, order=4):
        """d_k f_c of fields f [ncomp, N] (FP64; host or device) on this
        lattice -> CUDA tensor [3, ncomp, N], by the library's stencils."""
        torch = _torch()
        f = self._dev64(f, -1 if getattr(f, "ndim", 1) > 1 else 1)
        ncomp = f.shape[0]
        nb = ctypes.c_size_t(0)
        call("cslbm_lattice_gradient_scratch_bytes", self.ctx, ncomp, int(order), ctypes.byref(nb))
        scratch = torch.empty(max(nb.value, 8), dtype=torch.uint8, device=self.device)
        out = torch.empty((3, ncomp, self.N), dtype=torch.float64, device=self.device)
        call("cslbm_lattice_gradient", self.ctx, f.data_ptr(), ncomp, int(order), out.data_ptr(), scratch.data_ptr(),
             scratch.numel())
        self._hold(f, scratch)
        return out

    def _metric_scratch(self, order):
        torch = _torch()
        nb = ctypes.c_size_t(0)
        call("cslbm_metric_lattice_scratch_bytes", self.ctx, int(order), ctypes.byref(nb))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.device)

    def set_metric_lattice(self, g6, order=4):
        """set_metric with dg computed from g6 on the lattice."""
        g = self._dev64(g6, 6)
        scratch = self._metric_scratch(order)
        call("cslbm_set_metric_lattice", self.ctx, g.data_ptr(), int(order), scratch.data_ptr(), scratch.numel())
        self._hold(g, scratch)

    def update_metric_lattice(self, g6, J9, order=4):
        """update_metric (metric change + transformation) with dg from g6 on the lattice."""
        g = self._dev64(g6, 6)
        J = self._dev64(J9, 9)
        scratch = self._metric_scratch(order)
        call("cslbm_update_metric_lattice", self.ctx, g.data_ptr(), J.data_ptr(), int(order), scratch.data_ptr(),
             scratch.numel())
        self._hold(g, J, scratch)

    def set_chart(self, chart):
        """Metric and Jacobian of an inputs.Chart (no transformation)."""
        self.set_metric(chart.g6, chart.dg18)
        self.set_jacobian(chart.J9)

    # -- state --------------------------------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        p1, d1, k1 = self._arg(rho, self.N)
        p2, d2, k2 = self._arg(u, 3 * self.N)
        on_dev = d1 if rho is not None else d2
        call("cslbm_init_equilibrium", self.ctx, p1, p2, on_dev)

    def set_boundary_velocity(self, axis, side, u3):
        p, d, k = self._arg(u3, 3 * self.face_nodes(axis))
        call("cslbm_set_boundary_velocity", self.ctx, axis, side, p, d)

    def step(self, nsteps=1):
        call("cslbm_step", self.ctx, int(nsteps))

    def moments(self, cartesian=False, host=True):
        """(rho [N], u [3, N]) FP64 -- numpy arrays (host=True) or CUDA tensors."""
        if host:
            rho = np.empty(self.N)
            u = np.empty((3, self.N))
            call("cslbm_get_moments", self.ctx, rho.ctypes.data, u.ctypes.data, int(cartesian), 0)
            return rho, u
        torch = _torch()
        rho = torch.empty(self.N, dtype=torch.float64, device=self.device)
        u = torch.empty((3, self.N), dtype=torch.float64, device=self.device)
        call("cslbm_get_moments", self.ctx, rho.data_ptr(), u.data_ptr(), int(cartesian), 1)
        return rho, u

    def total_mass(self):
        out = ctypes.c_double(0.0)
        call("cslbm_total_mass", self.ctx, ctypes.byref(out))
        return out.value

    def total_mass_static(self):
        """Total mass without touching the workspace scratch or allocating
        (per-block partials in a fixed device array; see cslbm.h)."""
        out = ctypes.c_double(0.0)
        call("cslbm_total_mass_static", self.ctx, ctypes.byref(out))
        return out.value

    def wall_force(self, axis, side):
        out = (ctypes.c_double * 3)()
        call("cslbm_wall_force", self.ctx, axis, side, out)
        return np.array(out[:])

    def check(self):
        """True if the state is finite and subsonic; False on CSLBM_EUNSTABLE."""
        lib = _abi.load()
        st = lib.cslbm_check(self.ctx)
        if st == _abi.EUNSTABLE:
            return False
        if st != _abi.OK:
            raise _abi.CslbmError(st, "cslbm_check", lib.cslbm_last_error().decode())
        return True

    def state_bytes(self):
        n = ctypes.c_size_t(0)
        call("cslbm_state_bytes", self.ctx, ctypes.byref(n))
        return n.value

    def save_state(self):
        torch = _torch()
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        call("cslbm_save_state", self.ctx, buf.data_ptr(), buf.numel(), 1)
        return buf

    def load_state(self, buf):
        call("cslbm_load_state", self.ctx, buf.data_ptr(), buf.numel(), 1)

    def profile(self, enable=True):
        """Start (or stop) event timing of each LBM step and launch counting."""
        call("cslbm_profile_enable", self.ctx, int(bool(enable)))

    def profile_read(self):
        """(total ms of the profiled steps, number of steps, kernel launches)."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_longlong(0)
        k = ctypes.c_longlong(0)
        call("cslbm_profile_read", self.ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k))
        return ms.value, n.value, k.value

    def close(self):
        if getattr(self, "_owned", True) and getattr(self, "ctx", None) is not None and self.ctx.value:
            _abi.load().cslbm_destroy(self.ctx)
        self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @classmethod
    def _channel(cls, ctx, n, device, stream, owner):
        """A view of a context owned by a batch (not destroyed by this object)."""
        self = cls.__new__(cls)
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        self.device = device
        self.stream = stream
        self.ctx = ctx
        self._owned = False
        self._owner = owner
        return self


def _params(n, bc_lo, bc_hi, tau, theta, fext, storage, literal_a2, step_kernel):
    return _abi.Params((ctypes.c_int * 3)(*n), (ctypes.c_int * 3)(*bc_lo), (ctypes.c_int * 3)(*bc_hi), float(tau),
                       float(theta), (ctypes.c_double * 3)(*fext), STORAGE[storage], int(bool(literal_a2)),
                       STEP_KERNEL[step_kernel])


class CurvedBatch:
    """Independent FP32 channels of any sizes advanced together (two kernel
    launches per step for the whole batch, replayed from a CUDA graph).

    channels: list of dicts with keys n, bc_lo, bc_hi, tau and optionally
    fext, theta.  batch[i] is a CurvedLattice view of channel i (geometry,
    boundary velocities, initialisation, moments, forces work on it)."""

    def __init__(self, channels, device=None, stream=None):
        torch = _torch()
        _abi.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        nb = len(channels)
        arr = (_abi.Params * nb)()
        for i, ch in enumerate(channels):
            bc_hi = ch.get("bc_hi", ch["bc_lo"])
            arr[i] = _params(ch["n"], ch["bc_lo"], bc_hi, ch["tau"], ch.get("theta", 0.0),
                             ch.get("fext", (0.0, 0.0, 0.0)), "fp32", False, "flat")
        nbytes = ctypes.c_size_t(0)
        call("cslbm_batch_workspace_bytes", nb, arr, ctypes.byref(nbytes))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.batch = ctypes.c_void_p()
        call("cslbm_batch_create", nb, arr, self.workspace.data_ptr(), nbytes.value, self.stream.cuda_stream,
             ctypes.byref(self.batch))
        self.channels = []
        for i, ch in enumerate(channels):
            c = ctypes.c_void_p()
            call("cslbm_batch_context", self.batch, i, ctypes.byref(c))
            self.channels.append(CurvedLattice._channel(c, ch["n"], self.device, self.stream, self))
        self.nodes = sum(c.N for c in self.channels)

    def __len__(self):
        return len(self.channels)

    def __getitem__(self, i):
        return self.channels[i]

    def step(self, nsteps=1):
        call("cslbm_batch_step", self.batch, int(nsteps))

    def tune(self, reps=10):
        """Pick the tile shape (nodes per block, nodes per work item, blocks
        per SM) by timing the candidates on this batch; returns (chosen,
        {candidate: ms per step})."""
        shape = (ctypes.c_int * 3)()
        best = ctypes.c_float(0.0)
        call("cslbm_batch_tune", self.batch, int(reps), shape, ctypes.byref(best))
        n = ctypes.c_int(0)
        call("cslbm_batch_tune_results", self.batch, 0, None, None, ctypes.byref(n))
        shapes = (ctypes.c_int * (3 * n.value))()
        ms = (ctypes.c_float * n.value)()
        call("cslbm_batch_tune_results", self.batch, n.value, shapes, ms, ctypes.byref(n))
        table = {tuple(shapes[3 * i:3 * i + 3]): ms[i] for i in range(n.value)}
        return tuple(shape[:]), table

    def set_shape(self, shape):
        """Tile shape (nodes per block, nodes per work item, blocks per SM) by hand."""
        call("cslbm_batch_set_shape", self.batch, (ctypes.c_int * 3)(*shape))

    def check(self):
        """True unless a batch step's grid barrier ran out of time (cleared by this call)."""
        lib = _abi.load()
        st = lib.cslbm_batch_check(self.batch)
        if st == _abi.ETIMEOUT:
            return False
        if st != _abi.OK:
            raise _abi.CslbmError(st, "cslbm_batch_check", lib.cslbm_last_error().decode())
        return True

    def launches(self):
        k = ctypes.c_longlong(0)
        call("cslbm_batch_launches", self.batch, ctypes.byref(k))
        return k.value

    def close(self):
        if getattr(self, "batch", None) is not None and self.batch.value:
            for c in self.channels:
                c.ctx = ctypes.c_void_p()
            _abi.load().cslbm_batch_destroy(self.batch)
            self.batch = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CurvedLattice2D:
    """A D2Q9 lattice n = (n0, n1) carrying a metric field (the library's
    cslbm2d_* calls, one method each).  bc per axis as for CurvedLattice;
    storage "fp32" or "fp64"."""

    def __init__(self, n, bc_lo=(0, 0), bc_hi=None, tau=0.8, theta=0.0, fext=(0.0, 0.0), storage="fp32",
                 device=None, stream=None):
        torch = _torch()
        _abi.load()
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        bc_hi = bc_lo if bc_hi is None else bc_hi
        self.params = _abi.Params2D((ctypes.c_int * 2)(*self.n), (ctypes.c_int * 2)(*bc_lo),
                                    (ctypes.c_int * 2)(*bc_hi), float(tau), float(theta),
                                    (ctypes.c_double * 2)(*fext), STORAGE[storage])
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        nb = ctypes.c_size_t(0)
        call("cslbm2d_workspace_bytes", ctypes.byref(self.params), ctypes.byref(nb))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self.ctx = ctypes.c_void_p()
        call("cslbm2d_create", ctypes.byref(self.params), self.workspace.data_ptr(), nb.value,
             self.stream.cuda_stream, ctypes.byref(self.ctx))

    def _arg(self, a, count):
        """(pointer, on_device, keep-alive) for an FP64 input of `count` values
        (a CUDA tensor stays on the device; anything else is a host array)."""
        if a is None:
            return None, 1, None
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.device.type != "cuda":
                a = a.detach().to(torch.float64).contiguous().numpy()
            else:
                t = a.detach().to(self.device, torch.float64).contiguous()
                if t.numel() != count:
                    raise ValueError(f"expected {count} values, got {t.numel()}")
                t.record_stream(self.stream)  # a converted copy may be read after this call returns
                return t.data_ptr(), 1, t
        h = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        if h.size != count:
            raise ValueError(f"expected {count} values, got {h.size}")
        return h.ctypes.data, 0, h

    def set_metric(self, g3, dg6):
        p1, d1, k1 = self._arg(g3, 3 * self.N)
        p2, d2, k2 = self._arg(dg6, 6 * self.N)
        if d1 != d2:
            raise ValueError("g3 and dg6 must both be host or both device arrays")
        call("cslbm2d_set_metric", self.ctx, p1, p2, d1)

    def set_jacobian(self, J4):
        p, d, k = self._arg(J4, 4 * self.N)
        call("cslbm2d_set_jacobian", self.ctx, p, d)

    def set_chart(self, chart):
        self.set_metric(chart.g3, chart.dg6)
        self.set_jacobian(chart.J4)

    def update_metric(self, g3, dg6, J4):
        p1, d1, k1 = self._arg(g3, 3 * self.N)
        p2, d2, k2 = self._arg(dg6, 6 * self.N)
        p3, d3, k3 = self._arg(J4, 4 * self.N)
        if not (d1 == d2 == d3):
            raise ValueError("metric inputs must all be host or all device arrays")
        call("cslbm2d_update_metric", self.ctx, p1, p2, p3, d1)

    def set_boundary_velocity(self, axis, side, u2):
        p, d, k = self._arg(u2, 2 * self.n[1 - int(axis)]) if 0 <= int(axis) <= 1 else (None, 1, None)
        call("cslbm2d_set_boundary_velocity", self.ctx, int(axis), int(side), p, d)
        self._keep_face = getattr(self, "_keep_face", {})
        self._keep_face[(axis, side)] = k

    def init_equilibrium(self, rho=None, u=None):
        p1, d1, k1 = self._arg(rho, self.N)
        p2, d2, k2 = self._arg(u, 2 * self.N)
        on_dev = d1 if rho is not None else d2
        call("cslbm2d_init_equilibrium", self.ctx, p1, p2, on_dev)

    def step(self, nsteps=1):
        call("cslbm2d_step", self.ctx, int(nsteps))

    def moments(self, cartesian=False):
        rho = np.empty(self.N)
        u = np.empty((2, self.N))
        call("cslbm2d_get_moments", self.ctx, rho.ctypes.data, u.ctypes.data, int(cartesian), 0)
        return rho, u

    def total_mass(self):
        out = ctypes.c_double(0.0)
        call("cslbm2d_total_mass", self.ctx, ctypes.byref(out))
        return out.value

    def wall_force(self, axis, side):
        out = (ctypes.c_double * 2)()
        call("cslbm2d_wall_force", self.ctx, int(axis), int(side), out)
        return np.array(out[:])

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            _abi.load().cslbm2d_destroy(self.ctx)
        self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
