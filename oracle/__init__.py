"""FP64 CPU oracle of the curved-space lattice Boltzmann method (arXiv 1803.07822).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py`` -- never by the library.  It shares
no code with the CUDA path; see ``cslbm_oracle.c`` for the method as written
from the paper (literal f-form, Sec. II; geometry, App. A; Hermite
expansion, App. B; lattice gradient, App. D; transformation, Sec. IV.B).

Parity unpinned (no printed value to match; held only by convergence and
invariant tests): the sqrt(g) factor on the non-equilibrium part of the wall
rule.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cslbm_oracle.c")
_SRC2D = os.path.join(_HERE, "cslbm_oracle2d.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, WALL, INFLOW, OUTFLOW = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC2D))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, _SRC2D, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            for name in ("orc_geometry", "orc_init", "orc_step", "orc_fill_boundary",
                         "orc_moments", "orc_mass", "orc_wall_force", "orc_transform",
                         "orc_feq", "orc_forcing_recompose", "orc_forcing_moments",
                         "orc_lattice", "orc_lattice_gradient", "orc_lattice_laplacian",
                         "orc_transform_interp", "o2_lattice", "o2_geometry", "o2_init", "o2_step",
                         "o2_moments", "o2_mass", "o2_wall_force", "o2_transform", "o2_forcing_recompose",
                         "o2_forcing_moments"):
                getattr(_lib, name).restype = ctypes.c_int
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double),
                ("fext", ctypes.c_double * 3), ("literal_a2", ctypes.c_int)]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def lattice():
    """(c [19,3] int, w [19]) as the oracle defines them."""
    lib = _load()
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    lib.orc_lattice(_p(c), _p(w))
    return c.reshape(19, 3), w


def _field_params(n, bc_lo, bc_hi):
    p = _Params()
    p.n[:] = list(n)
    p.bc_lo[:] = list(bc_lo)
    p.bc_hi[:] = list(bc_lo if bc_hi is None else bc_hi)
    p.tau, p.theta = 1.0, 1.0 / 3.0
    return p


def lattice_gradient(n, f, order=2, bc_lo=(0, 0, 0), bc_hi=None):
    """d_k f_c of ncomp fields f [ncomp, N] -> [3, ncomp, N] by the isotropic
    D3Q19 stencils of App. D, order 2 or 4; non-periodic faces continue the
    field polynomially (degree = order)."""
    f = _f64(f)
    f2 = f.reshape(-1, int(np.prod(n)))
    out = np.zeros((3, f2.shape[0], f2.shape[1]))
    p = _field_params(n, bc_lo, bc_hi)
    if _load().orc_lattice_gradient(ctypes.byref(p), _p(f2), f2.shape[0], int(order), _p(out)):
        raise ValueError("orc_lattice_gradient: bad order or too few nodes on a non-periodic axis")
    return out


def lattice_laplacian(n, f, order=2, bc_lo=(0, 0, 0), bc_hi=None):
    """L f_c = (2/c_s^2) sum_l w_l (f(x + c_l) - f(x)) of f [ncomp, N] (App. D)."""
    f2 = _f64(f).reshape(-1, int(np.prod(n)))
    out = np.zeros_like(f2)
    p = _field_params(n, bc_lo, bc_hi)
    if _load().orc_lattice_laplacian(ctypes.byref(p), _p(f2), f2.shape[0], int(order), _p(out)):
        raise ValueError("orc_lattice_laplacian: bad order")
    return out


def geometry(n, g6, dg18):
    """g_ij, d_k g_ij -> (sqrt g [N], g^ij [9,N], Gamma^i_jk [27,N])."""
    lib = _load()
    N = int(np.prod(n))
    g6 = _f64(g6, (6, N))
    dg18 = _f64(dg18, (18, N))
    sg = np.zeros(N)
    gi = np.zeros((9, N))
    gam = np.zeros((27, N))
    nn = (ctypes.c_int * 3)(*n)
    if lib.orc_geometry(nn, _p(g6), _p(dg18), _p(sg), _p(gi), _p(gam)) != 0:
        raise ValueError("metric not positive definite")
    return sg, gi, gam


def feq(rho, j3, ginv9, sqrtg, theta=1.0 / 3.0):
    lib = _load()
    j3 = _f64(j3)
    gi = _f64(ginv9)
    out = np.zeros(19)
    lib.orc_feq(ctypes.c_double(rho), _p(j3), _p(gi), ctypes.c_double(sqrtg),
                ctypes.c_double(theta), _p(out))
    return out


def forcing_recompose(A, B3, C9, sqrtg):
    lib = _load()
    B3 = _f64(B3)
    C9 = _f64(C9)
    out = np.zeros(19)
    lib.orc_forcing_recompose(ctypes.c_double(A), _p(B3), _p(C9), ctypes.c_double(sqrtg), _p(out))
    return out


def forcing_moments(j3, T9, Dj9, ginv9, gam27, theta=1.0 / 3.0, fext3=(0, 0, 0)):
    """A, B^i, C^ij (Eqs. forcing-A/B/C) for one node; Dj9[k*3+i] = d_k(rho u^i)."""
    lib = _load()
    args = [_f64(x) for x in (j3, T9, Dj9, ginv9, gam27)]
    fe = _f64(fext3)
    A = ctypes.c_double(0.0)
    B = np.zeros(3)
    C = np.zeros(9)
    lib.orc_forcing_moments(*[_p(a) for a in args], ctypes.c_double(theta), _p(fe),
                            ctypes.byref(A), _p(B), _p(C))
    return A.value, B, C


class Lattice:
    """One channel advanced by the oracle.

    n = (n0, n1, n2), axis 0 fastest; bc_lo/bc_hi per axis in
    {PERIODIC, WALL, INFLOW, OUTFLOW}; fext is the contravariant body force
    density (constant); theta defaults to c_s^2 = 1/3.
    """

    def __init__(self, n, bc_lo=(0, 0, 0), bc_hi=None, tau=0.8, theta=1.0 / 3.0,
                 fext=(0.0, 0.0, 0.0), literal_a2=False):
        self.lib = _load()
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        bc_hi = bc_lo if bc_hi is None else bc_hi
        self.params = _Params((ctypes.c_int * 3)(*self.n), (ctypes.c_int * 3)(*bc_lo),
                              (ctypes.c_int * 3)(*bc_hi), float(tau), float(theta),
                              (ctypes.c_double * 3)(*fext), int(bool(literal_a2)))
        self.f = np.zeros((19, self.N))
        self.Fprev = np.zeros((19, self.N))
        self.sqrtg = np.ones(self.N)
        gi = np.zeros((9, self.N))
        gi[[0, 4, 8]] = 1.0
        self.ginv = gi
        self.gam = np.zeros((27, self.N))
        self._faces = [None] * 6
        self._face_ptrs = (ctypes.c_void_p * 6)()

    # -- geometry and boundary data ------------------------------------
    def set_metric(self, g6, dg18):
        self.sqrtg, self.ginv, self.gam = geometry(self.n, g6, dg18)

    def face_shape(self, axis):
        o = sorted(((axis + 1) % 3, (axis + 2) % 3))
        return self.n[o[0]] * self.n[o[1]]

    def set_face_velocity(self, axis, side, u3):
        """Contravariant velocity [3, face nodes] imposed on face (axis, side)."""
        k = axis * 2 + side
        if u3 is None:
            self._faces[k] = None
            self._face_ptrs[k] = None
        else:
            a = _f64(u3, (3, self.face_shape(axis)))
            self._faces[k] = a
            self._face_ptrs[k] = a.ctypes.data

    def _check(self, rc, what):
        if rc != 0:
            raise ValueError(f"oracle {what} failed ({rc})")

    # -- method ---------------------------------------------------------
    def init(self, rho0=None, u0=None):
        rho0 = np.ones(self.N) if rho0 is None else _f64(rho0, (self.N,))
        u0 = np.zeros((3, self.N)) if u0 is None else _f64(u0, (3, self.N))
        self._check(self.lib.orc_init(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv),
                                      _p(self.gam), _p(rho0), _p(u0), self._face_ptrs,
                                      _p(self.f), _p(self.Fprev)), "init")

    def step(self, nsteps=1):
        self._check(self.lib.orc_step(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv),
                                      _p(self.gam), self._face_ptrs, _p(self.f), _p(self.Fprev),
                                      ctypes.c_int(nsteps)), "step")

    def filled(self):
        fb = np.zeros_like(self.f)
        self._check(self.lib.orc_fill_boundary(ctypes.byref(self.params), _p(self.sqrtg),
                                               _p(self.ginv), self._face_ptrs, _p(self.f),
                                               _p(fb)), "fill")
        return fb

    def moments(self, J9=None):
        """(rho [N], u [3,N]) -- contravariant, or Cartesian v = J u with J9."""
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        Jkeep = None if J9 is None else _f64(J9, (9, self.N))
        Jp = None if Jkeep is None else _p(Jkeep)
        self._check(self.lib.orc_moments(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv),
                                         self._face_ptrs, _p(self.f), Jp, _p(rho), _p(u)),
                    "moments")
        return rho, u

    def mass(self):
        m = ctypes.c_double(0.0)
        self._check(self.lib.orc_mass(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv),
                                      self._face_ptrs, _p(self.f), ctypes.byref(m)), "mass")
        return m.value

    def wall_force(self, axis, side, J9):
        J = _f64(J9, (9, self.N))
        out = np.zeros(3)
        self._check(self.lib.orc_wall_force(ctypes.byref(self.params), _p(self.sqrtg),
                                            _p(self.ginv), self._face_ptrs, _p(self.f), _p(J),
                                            ctypes.c_int(axis), ctypes.c_int(side), _p(out)),
                    "wall_force")
        return out

    def transform(self, g6_new, dg18_new, Jold9, Jnew9):
        """Chart change (Sec. IV.B): transform f and the forcing history, then
        adopt the new geometry."""
        sg_new, gi_new, gam_new = geometry(self.n, g6_new, dg18_new)
        Jo = _f64(Jold9, (9, self.N))
        Jn = _f64(Jnew9, (9, self.N))
        self._check(self.lib.orc_transform(ctypes.byref(self.params), _p(self.sqrtg),
                                           _p(self.ginv), _p(sg_new), _p(Jo), _p(Jn),
                                           self._face_ptrs, _p(self.f), _p(self.Fprev)),
                    "transform")
        self.sqrtg, self.ginv, self.gam = sg_new, gi_new, gam_new

    def transform_interp(self, g6_new, dg18_new, Jold9, Jnew9, psi3):
        """Chart change with interpolation (Sec. IV.B): every new node takes the
        old moments at psi3 [3, N] (old lattice coordinates of its point),
        trilinearly, then transforms them with J~^-1 J(psi) and recomposes."""
        sg_new, gi_new, gam_new = geometry(self.n, g6_new, dg18_new)
        Jo = _f64(Jold9, (9, self.N))
        Jn = _f64(Jnew9, (9, self.N))
        ps = _f64(psi3, (3, self.N))
        self._check(self.lib.orc_transform_interp(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv),
                                                  _p(sg_new), _p(Jo), _p(Jn), _p(ps), self._face_ptrs,
                                                  _p(self.f), _p(self.Fprev)), "transform_interp")
        self.sqrtg, self.ginv, self.gam = sg_new, gi_new, gam_new


# ---------------------------------------------------------------------------
# two dimensions (D2Q9), cslbm_oracle2d.c
# ---------------------------------------------------------------------------
class _Params2(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 2), ("bc_lo", ctypes.c_int * 2), ("bc_hi", ctypes.c_int * 2),
                ("tau", ctypes.c_double), ("theta", ctypes.c_double), ("fext", ctypes.c_double * 2)]


def lattice2d():
    """(c [9,2] int, w [9]) of the D2Q9 oracle."""
    c = np.zeros(18, dtype=np.int32)
    w = np.zeros(9)
    _load().o2_lattice(_p(c), _p(w))
    return c.reshape(9, 2), w


def forcing_recompose2d(A, B2, C4, sqrtg):
    """F_l [9] of one node from its forcing moments A, B [2], C [2x2] (Eq. forcing2 in 2-D)."""
    out = np.zeros(9)
    Bk, Ck = _f64(B2, (2,)), _f64(C4, (4,))
    _load().o2_forcing_recompose(ctypes.c_double(A), _p(Bk), _p(Ck), ctypes.c_double(sqrtg), _p(out))
    return out


def forcing_moments2d(j2, T4, Dj4, ginv4, gam8, theta=1.0 / 3.0, fext2=(0, 0)):
    """A, B^i, C^ij (Eqs. forcing-A/B/C in 2-D) for one node; Dj4[k*2+i] = d_k(rho u^i)."""
    args = [_f64(x) for x in (j2, T4, Dj4, ginv4, gam8)]
    fe = _f64(fext2)
    A = ctypes.c_double(0.0)
    B = np.zeros(2)
    C = np.zeros(4)
    _load().o2_forcing_moments(*[_p(a) for a in args], ctypes.c_double(theta), _p(fe), ctypes.byref(A), _p(B),
                               _p(C))
    return A.value, B, C


def geometry2d(n, g3, dg6):
    """g_ij [3, N], d_k g_ij [6, N] -> (sqrt g [N], g^ij [4, N], Gamma^i_jk [8, N])."""
    N = int(np.prod(n))
    g3, dg6 = _f64(g3, (3, N)), _f64(dg6, (6, N))
    sg, gi, gam = np.zeros(N), np.zeros((4, N)), np.zeros((8, N))
    if _load().o2_geometry((ctypes.c_int * 2)(*n), _p(g3), _p(dg6), _p(sg), _p(gi), _p(gam)):
        raise ValueError("metric not positive definite")
    return sg, gi, gam


class Lattice2D:
    """The D2Q9 oracle: literal f-form, FP64, n = (n0, n1), bc per axis."""

    def __init__(self, n, bc_lo=(0, 0), bc_hi=None, tau=0.8, theta=1.0 / 3.0, fext=(0.0, 0.0)):
        self.lib = _load()
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        bc_hi = bc_lo if bc_hi is None else bc_hi
        self.params = _Params2((ctypes.c_int * 2)(*self.n), (ctypes.c_int * 2)(*bc_lo), (ctypes.c_int * 2)(*bc_hi),
                               float(tau), float(theta), (ctypes.c_double * 2)(*fext))
        self.f = np.zeros((9, self.N))
        self.Fprev = np.zeros((9, self.N))
        self.sqrtg = np.ones(self.N)
        self.ginv = np.zeros((4, self.N))
        self.ginv[[0, 3]] = 1.0
        self.gam = np.zeros((8, self.N))
        self._faces = [None] * 4
        self._face_ptrs = (ctypes.c_void_p * 4)()

    def set_metric(self, g3, dg6):
        self.sqrtg, self.ginv, self.gam = geometry2d(self.n, g3, dg6)

    def set_face_velocity(self, axis, side, u2):
        k = axis * 2 + side
        if u2 is None:
            self._faces[k], self._face_ptrs[k] = None, None
        else:
            a = _f64(u2, (2, self.n[1 - axis]))
            self._faces[k] = a
            self._face_ptrs[k] = a.ctypes.data

    def _check(self, rc, what):
        if rc:
            raise ValueError(f"oracle {what} failed")

    def init(self, rho0=None, u0=None):
        rho0 = np.ones(self.N) if rho0 is None else _f64(rho0, (self.N,))
        u0 = np.zeros((2, self.N)) if u0 is None else _f64(u0, (2, self.N))
        self._check(self.lib.o2_init(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), _p(self.gam), _p(rho0),
                                     _p(u0), self._face_ptrs, _p(self.f), _p(self.Fprev)), "init")

    def step(self, nsteps=1):
        self._check(self.lib.o2_step(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), _p(self.gam),
                                     self._face_ptrs, _p(self.f), _p(self.Fprev), int(nsteps)), "step")

    def moments(self, J4=None):
        rho, u = np.zeros(self.N), np.zeros((2, self.N))
        Jk = None if J4 is None else _f64(J4, (4, self.N))
        self._check(self.lib.o2_moments(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), self._face_ptrs,
                                        _p(self.f), None if Jk is None else _p(Jk), _p(rho), _p(u)), "moments")
        return rho, u

    def mass(self):
        out = ctypes.c_double(0.0)
        self._check(self.lib.o2_mass(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), self._face_ptrs,
                                     _p(self.f), ctypes.byref(out)), "mass")
        return out.value

    def wall_force(self, axis, side, J4):
        out = np.zeros(2)
        Jk = _f64(J4, (4, self.N))
        self._check(self.lib.o2_wall_force(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), self._face_ptrs,
                                           _p(self.f), _p(Jk), int(axis), int(side), _p(out)), "wall force")
        return out

    def transform(self, g3_new, dg6_new, Jold4, Jnew4):
        sg, gi, gam = geometry2d(self.n, g3_new, dg6_new)
        Jo, Jn = _f64(Jold4, (4, self.N)), _f64(Jnew4, (4, self.N))
        self._check(self.lib.o2_transform(ctypes.byref(self.params), _p(self.sqrtg), _p(self.ginv), _p(sg), _p(Jo),
                                          _p(Jn), self._face_ptrs, _p(self.f), _p(self.Fprev)), "transform")
        self.sqrtg, self.ginv, self.gam = sg, gi, gam
