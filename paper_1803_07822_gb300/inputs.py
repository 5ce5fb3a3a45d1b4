"""Seeded synthetic inputs: charts, metrics, boundary velocities, body forces.

This module serves both the CUDA path and the CPU oracle.  It holds no step of
the lattice Boltzmann method: it only plays the part of the caller -- the FEM
shell of the paper, which is out of scope -- that hands the solver a chart
h(x) and the metric it induces.  All geometry is analytic and FP64.

Conventions: a field on an (n0, n1, n2) lattice is an array [components, N]
with node = x + n0*(y + n1*z) (axis 0 fastest).  J9[a*3+i] = d h^a / d x^i.
g6 holds g_00, g_01, g_02, g_11, g_12, g_22; dg18[k*6+ij] = d_k g_ij.

Channel layout: a channel is described by (wall, span, flow) axes.  The
default layout puts the wall-normal direction on axis 2 (walls at x2 = 0 and
x2 = n2-1; the x2 = 0 wall is fixed), the flow direction on axis 1 and the
periodic span on axis 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SYM = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def grid(n):
    """Coordinate arrays (x, y, z), each [N], in node order."""
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)


@dataclass
class Chart:
    """A chart h: lattice -> Cartesian space, given by its first and second
    derivatives at the nodes, with the metric it induces (g = J^T J)."""
    n: tuple
    J9: np.ndarray          # [9, N]
    hess: np.ndarray        # [27, N]  d_j d_k h^a at (a*9 + j*3 + k)
    g6: np.ndarray = field(init=False)
    dg18: np.ndarray = field(init=False)

    def __post_init__(self):
        N = self.J9.shape[1]
        J = self.J9.reshape(3, 3, N)            # [a, i]
        Hs = self.hess.reshape(3, 3, 3, N)      # [a, j, k]
        g = np.einsum("ain,ajn->ijn", J, J)
        dg = np.einsum("akin,ajn->kijn", Hs, J) + np.einsum("ain,akjn->kijn", J, Hs)
        self.g6 = np.stack([g[i, j] for i, j in SYM])
        self.dg18 = np.stack([dg[k, i, j] for k in range(3) for i, j in SYM])

    @property
    def N(self):
        return self.J9.shape[1]


def flat_chart(n):
    N = int(np.prod(n))
    J9 = np.zeros((9, N))
    J9[[0, 4, 8]] = 1.0
    return Chart(tuple(n), J9, np.zeros((27, N)))


def reparam_chart(n, eps):
    """Pure re-parametrisation of a flat channel across axis 0:
    x_c = x + eps * L/pi * sin(pi x / L), L = n0 - 1 (end points fixed).
    Space stays flat; only the coordinates are stretched."""
    x, _, _ = grid(n)
    L = n[0] - 1
    N = x.size
    J9 = np.zeros((9, N))
    J9[0] = 1.0 + eps * np.cos(np.pi * x / L)
    J9[4] = 1.0
    J9[8] = 1.0
    hess = np.zeros((27, N))
    hess[0] = -eps * (np.pi / L) * np.sin(np.pi * x / L)
    return Chart(tuple(n), J9, hess)


def reparam_position(n, eps):
    """Cartesian wall-normal coordinate x_c(x) of the nodes of reparam_chart."""
    x, _, _ = grid(n)
    L = n[0] - 1
    return x + eps * L / np.pi * np.sin(np.pi * x / L)


def annulus_chart(n, r0):
    """Polar chart of the gap between two concentric cylinders (lattice
    units): axis 0 radial, r = r0 + x; axis 1 around the cylinders, theta =
    y / r0 (unit arc at the inner cylinder, periodic for a flow that does not
    depend on theta); axis 2 along them.  Flat space in curved coordinates,
    g = diag(1, (r / r0)^2, 1)."""
    x, y, _ = grid(n)
    r, th = r0 + x, y / r0
    c, s = np.cos(th), np.sin(th)
    N = x.size
    J9 = np.zeros((9, N))
    J9[0], J9[1] = c, -(r / r0) * s
    J9[3], J9[4] = s, (r / r0) * c
    J9[8] = 1.0
    hess = np.zeros((27, N))  # d_j d_k h^a at a*9 + j*3 + k
    hess[0 * 9 + 0 * 3 + 1] = hess[0 * 9 + 1 * 3 + 0] = -s / r0
    hess[0 * 9 + 1 * 3 + 1] = -(r / r0 ** 2) * c
    hess[1 * 9 + 0 * 3 + 1] = hess[1 * 9 + 1 * 3 + 0] = c / r0
    hess[1 * 9 + 1 * 3 + 1] = -(r / r0 ** 2) * s
    return Chart(tuple(n), J9, hess)


@dataclass
class Deformation:
    """Wall displacement d(p, s) of the top wall and its derivatives, per node
    (the same value for every wall-normal index)."""
    d: np.ndarray
    dp: np.ndarray
    ds: np.ndarray
    dpp: np.ndarray
    dps: np.ndarray
    dss: np.ndarray

    def scaled(self, a):
        return Deformation(*(a * v for v in (self.d, self.dp, self.ds, self.dpp, self.dps, self.dss)))


LAYOUT = (2, 0, 1)  # (wall-normal axis, span axis, flow axis)


def fourier_deformation(n, n_modes, amp, seed, flow_periodic=True, kmax=4, lmax=3,
                        coeffs=None, modes=None, layout=LAYOUT):
    """d = amp * H * D / max|D| with D = sum_m c_m cos(2 pi k_m s/L_s + 2 pi l_m p/L_p + phi_m);
    on a non-periodic flow axis d is tapered by sin^2(pi s/(n_flow-1)) so that
    the inlet and outlet stay flat.  p and s are the span and flow coordinates
    of ``layout`` = (wall, span, flow) axes; H = n_wall - 1.  c_m ~ N(0,1), k_m in 1..kmax, l_m in 0..lmax,
    phi_m ~ U[0, 2 pi), all from numpy's default_rng(seed).  When ``coeffs`` and
    ``modes`` are given they replace the draws (``amp`` is then an absolute
    scale: d = amp * H * D)."""
    ax_w, ax_p, ax_s = layout
    r = grid(n)
    p, s = r[ax_p], r[ax_s]
    H = n[ax_w] - 1
    Ls = n[ax_s] if flow_periodic else n[ax_s] - 1
    Lp = n[ax_p]
    if modes is None:
        rng = np.random.default_rng(seed)
        k = rng.integers(1, kmax + 1, size=n_modes)
        l = rng.integers(0, lmax + 1, size=n_modes)
        c = rng.standard_normal(n_modes)
        phi = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    else:
        k, l, phi = (np.asarray(v, dtype=np.float64) for v in modes)
        c = np.asarray(coeffs, dtype=np.float64)
    D = np.zeros_like(s)
    Dp, Ds, Dpp, Dps, Dss = (np.zeros_like(s) for _ in range(5))
    for m in range(len(c)):
        ks = 2.0 * np.pi * k[m] / Ls
        lp = 2.0 * np.pi * l[m] / Lp
        th = ks * s + lp * p + phi[m]
        cth, sth = np.cos(th), np.sin(th)
        D += c[m] * cth
        Ds -= c[m] * ks * sth
        Dp -= c[m] * lp * sth
        Dss -= c[m] * ks * ks * cth
        Dpp -= c[m] * lp * lp * cth
        Dps -= c[m] * ks * lp * cth
    K = amp * H / np.max(np.abs(D)) if modes is None else amp * H
    if flow_periodic:
        S, S1, S2 = np.ones_like(s), np.zeros_like(s), np.zeros_like(s)
    else:
        w = np.pi / (n[ax_s] - 1)
        S = np.sin(w * s) ** 2
        S1 = w * np.sin(2.0 * w * s)
        S2 = 2.0 * w * w * np.cos(2.0 * w * s)
    return Deformation(K * D * S, K * Dp * S, K * (Ds * S + D * S1), K * Dpp * S,
                       K * (Dps * S + Dp * S1), K * (Dss * S + 2.0 * Ds * S1 + D * S2))


def channel_chart(n, dfm: Deformation, layout=LAYOUT):
    """Exterior linear interpolation between the fixed wall x_w = 0 and the
    displaced wall x_w = H (Sec. IV.A position coupling, case (i)):
    h^w = x_w (1 + d(p,s)/H), the other components the identity."""
    w, a_p, a_s = layout
    r = grid(n)
    xw = r[w]
    H = n[w] - 1
    N = xw.size
    J9 = np.zeros((9, N))
    J9[[0, 4, 8]] = 1.0
    J9[w * 3 + w] = 1.0 + dfm.d / H
    J9[w * 3 + a_p] = xw * dfm.dp / H
    J9[w * 3 + a_s] = xw * dfm.ds / H
    hess = np.zeros((27, N))

    def put(j, k, val):  # d_j d_k h^w
        hess[w * 9 + j * 3 + k] = val
        hess[w * 9 + k * 3 + j] = val

    put(w, a_p, dfm.dp / H)
    put(w, a_s, dfm.ds / H)
    put(a_p, a_p, xw * dfm.dpp / H)
    put(a_p, a_s, xw * dfm.dps / H)
    put(a_s, a_s, xw * dfm.dss / H)
    return Chart(tuple(n), J9, hess)


def face_nodes(n, axis, side):
    """Node indices of face (axis, side) in face order (the other two axes,
    lower axis fastest)."""
    x, y, z = grid(n)
    r = (x, y, z)
    sel = r[axis] == (n[axis] - 1 if side else 0)
    return np.nonzero(sel)[0]


def contravariant(J9, v3, nodes):
    """u = J^-1 v at the given nodes (Eq. vector_transform from C to Q)."""
    J = J9[:, nodes].T.reshape(-1, 3, 3)
    return np.linalg.solve(J, v3.T[..., None])[..., 0].T


def wall_velocity(n, chart: Chart, dfm_rate: Deformation, layout=LAYOUT):
    """Contravariant velocity of the displaced wall (x_w = n_w - 1) moving with
    d'(t): Cartesian v = dd/dt along the wall normal, u = J^-1 v."""
    w = layout[0]
    nodes = face_nodes(n, w, 1)
    v = np.zeros((3, nodes.size))
    v[w] = dfm_rate.d[nodes]
    return contravariant(chart.J9, v, nodes)


def inflow_profile(n, chart: Chart, umax, layout=LAYOUT):
    """Parabolic inflow on face (flow axis, low): Cartesian v_flow =
    4 umax xc (H - xc) / H^2 with xc the Cartesian wall-normal position."""
    w, _, a_s = layout
    nodes = face_nodes(n, a_s, 0)
    xw = grid(n)[w]
    H = n[w] - 1
    xc = xw[nodes] * chart.J9[w * 3 + w, nodes]  # h^w = x_w (1 + d/H), J^w_w = 1 + d/H
    v = np.zeros((3, nodes.size))
    v[a_s] = 4.0 * umax * xc * (H - xc) / (H * H)
    return contravariant(chart.J9, v, nodes)


def body_force(nu, umax, H):
    """Poiseuille drive: |F| = 8 nu umax / H^2 (centre-line speed umax)."""
    return 8.0 * nu * umax / (H * H)


def random_spd_metric(rng, eps=0.2):
    """A random symmetric positive-definite 3x3 metric near the identity."""
    A = np.eye(3) + eps * rng.standard_normal((3, 3))
    return A.T @ A


def time_law(t, period=2000.0):
    """Amplitude factor a(t) = sin^2(pi t / period) and its rate."""
    w = np.pi / period
    return np.sin(w * t) ** 2, w * np.sin(2.0 * w * t)


# --------------------------------------------------------------------------
# Workloads.  Each returns a dict with: n, bc_lo, bc_hi, tau, fext, chart and,
# where relevant, the deformation generator and the face velocities.
# --------------------------------------------------------------------------
WALL, PERIODIC, INFLOW, OUTFLOW = 1, 0, 2, 3


def _bcs(layout, flow_rule_lo, flow_rule_hi):
    lo, hi = [PERIODIC] * 3, [PERIODIC] * 3
    w, _, a_s = layout
    lo[w] = hi[w] = WALL
    lo[a_s], hi[a_s] = flow_rule_lo, flow_rule_hi
    return tuple(lo), tuple(hi)


def periodic_channel(n, tau, umax, n_modes, amp, seed, modes=None, coeffs=None, layout=LAYOUT, kmax=4, lmax=3):
    """Walls across the wall axis, periodic span and flow, body-force drive
    along the flow axis with centre-line speed umax."""
    nu = (tau - 0.5) / 3.0
    w, _, a_s = layout
    H = n[w] - 1
    dfm = fourier_deformation(n, n_modes, amp, seed, flow_periodic=True, kmax=kmax, lmax=lmax, modes=modes,
                              coeffs=coeffs, layout=layout)
    lo, hi = _bcs(layout, PERIODIC, PERIODIC)
    fext = [0.0, 0.0, 0.0]
    fext[a_s] = body_force(nu, umax, H)
    return dict(n=tuple(n), bc_lo=lo, bc_hi=hi, tau=tau, fext=tuple(fext), dfm=dfm,
                chart=channel_chart(n, dfm, layout), faces={}, layout=layout, wall_axis=w)


def fourier_modes(kmax, lmax, kmin=1):
    """The (k, l) pairs k in kmin..kmax along the flow, l in 0..lmax across,
    phase 0: one deformation coefficient per pair."""
    k, l = np.meshgrid(np.arange(kmin, kmax + 1), np.arange(0, lmax + 1), indexing="ij")
    return k.ravel().astype(float), l.ravel().astype(float), np.zeros(k.size)


def adjoint_channel(n=(64, 128, 64), kmax=8, lmax=3, seed=5000, tau=0.8, shrink=4.0, umax=0.05, layout=LAYOUT):
    """Periodic channel whose top-wall displacement is
    d = H / (shrink sqrt(M)) sum_m c_m cos(2 pi k_m s / L_s + 2 pi l_m p / L_p),
    M = (kmax) (lmax + 1) coefficients c_m ~ N(0, 0.02) from `seed`; body-force
    drive for centre-line speed umax.  The defaults (64 x 128 x 64, 32
    coefficients, shrink 4) keep the largest wall slope at 0.25."""
    modes = fourier_modes(kmax, lmax)
    M = len(modes[0])
    c = np.random.default_rng(seed).normal(0.0, 0.02, M)
    base = periodic_channel(n, tau, umax, 1, 0.0, 0, layout=layout)  # faces and drive
    return dict(n=tuple(n), modes=modes, c=c, scale=1.0 / (shrink * np.sqrt(M)), tau=tau, bc_lo=base["bc_lo"],
                bc_hi=base["bc_hi"], fext=base["fext"], layout=layout)


def tg_chart(n, t, eps=0.1, eta=0.05):
    """Periodic, separable, time-dependent chart of the Taylor-Green study:
    x_c^i = x^i - eps (L_i / 2 pi) cos(2 pi x^i / L_i - eta t) on the two
    in-plane axes (0, 1), the identity on axis 2; so J^i_i = 1 + eps sin(2 pi
    x^i / L_i - eta t) and g = diag(J00^2, J11^2, 1)."""
    r = grid(n)
    N = r[0].size
    J9 = np.zeros((9, N))
    hess = np.zeros((27, N))
    J9[8] = 1.0
    for a in (0, 1):
        k = 2 * np.pi / n[a]
        th = k * r[a] - eta * t
        J9[a * 3 + a] = 1.0 + eps * np.sin(th)
        hess[a * 9 + a * 3 + a] = eps * k * np.cos(th)
    return Chart(tuple(n), J9, hess)


def tg_position(n, t, eps=0.1, eta=0.05):
    """Cartesian positions x_c [3, N] of the nodes under tg_chart at time t."""
    r = grid(n)
    out = np.stack(r).astype(np.float64)
    for a in (0, 1):
        L = n[a]
        out[a] = r[a] - eps * (L / (2 * np.pi)) * np.cos(2 * np.pi * r[a] / L - eta * t)
    return out


def tg_psi(n, t_old, t_new, eps=0.1, eta=0.05):
    """Transition map psi = h_old^-1(h_new(x~)) [3, N] of tg_chart from t_old to
    t_new: per in-plane axis the solution x of x - eps (L/2pi) cos(2 pi x/L -
    eta t_old) = x_c(x~, t_new), by Newton's method (the map is monotone for
    eps < 1)."""
    xc = tg_position(n, t_new, eps, eta)
    r = grid(n)
    psi = np.stack(r).astype(np.float64)
    for a in (0, 1):
        L = n[a]
        k = 2 * np.pi / L
        x = xc[a].copy()
        for _ in range(50):
            fx = x - eps / k * np.cos(k * x - eta * t_old) - xc[a]
            dx = fx / (1.0 + eps * np.sin(k * x - eta * t_old))
            x -= dx
            if np.abs(dx).max() < 1e-14:
                break
        psi[a] = x
    return psi


def tg_velocity(xc, L, v0, nu, t):
    """The decaying 2D Taylor-Green field at Cartesian points xc [3, N]:
    v = v0 exp(-2 nu k^2 t) (sin kx cos ky, -cos kx sin ky, 0), k = 2 pi / L,
    and the density 1 - (v0^2 e^{-4 nu k^2 t} / (4 c_s^2)) (cos 2kx + cos 2ky)
    of its pressure."""
    k = 2 * np.pi / L
    d = np.exp(-2 * nu * k * k * t)
    v = np.zeros_like(xc)
    v[0] = v0 * d * np.sin(k * xc[0]) * np.cos(k * xc[1])
    v[1] = -v0 * d * np.cos(k * xc[0]) * np.sin(k * xc[1])
    rho = 1.0 - (v0 * d) ** 2 * 3.0 / 4.0 * (np.cos(2 * k * xc[0]) + np.cos(2 * k * xc[1]))
    return rho, v


# ---------------------------------------------------------------------------
# two dimensions (D2Q9): node = x + n0 y; g3 = (g00, g01, g11); dg6 = d_k g_ij
# at (k * 3 + ij); J4 = J^a_i at (a * 2 + i)
# ---------------------------------------------------------------------------
@dataclass
class Chart2D:
    n: tuple
    J4: np.ndarray    # [4, N]
    hess: np.ndarray  # [8, N] d_j d_k h^a at (a * 4 + j * 2 + k)

    @property
    def g3(self):
        J = self.J4.reshape(2, 2, -1)
        g = np.einsum("ain,ajn->ijn", J, J)
        return np.stack([g[0, 0], g[0, 1], g[1, 1]])

    @property
    def dg6(self):
        J = self.J4.reshape(2, 2, -1)
        Hs = self.hess.reshape(2, 2, 2, -1)  # [a, j, k]
        dg = np.einsum("akin,ajn->kijn", Hs, J) + np.einsum("ain,akjn->kijn", J, Hs)
        return np.stack([dg[k, i, j] for k in range(2) for i, j in ((0, 0), (0, 1), (1, 1))])


def grid2d(n):
    y, x = np.meshgrid(np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64)


def channel_chart2d(n, d, dd, ddd):
    """Exterior chart of a 2-D channel whose top wall (y = H = n1 - 1) is
    displaced by d(x): h^x = x, h^y = y (1 + d(x)/H); d, d', d'' per node."""
    x, y = grid2d(n)
    H = n[1] - 1
    N = x.size
    J4 = np.zeros((4, N))
    J4[0] = 1.0
    J4[2] = y * dd / H
    J4[3] = 1.0 + d / H
    hess = np.zeros((8, N))
    hess[4 + 0] = y * ddd / H      # d_x d_x h^y
    hess[4 + 1] = dd / H           # d_x d_y h^y
    hess[4 + 2] = dd / H           # d_y d_x h^y
    return Chart2D(tuple(n), J4, hess)


def flat_chart2d(n):
    N = int(np.prod(n))
    J4 = np.zeros((4, N))
    J4[[0, 3]] = 1.0
    return Chart2D(tuple(n), J4, np.zeros((8, N)))


def reparam_chart2d(n, eps):
    """Flat channel reparametrised across the walls (axis 1): y_c = y + eps (L/pi) sin(pi y / L), L = n1 - 1."""
    x, y = grid2d(n)
    L = n[1] - 1
    N = x.size
    J4 = np.zeros((4, N))
    J4[0] = 1.0
    J4[3] = 1.0 + eps * np.cos(np.pi * y / L)
    hess = np.zeros((8, N))
    hess[4 + 3] = -eps * np.pi / L * np.sin(np.pi * y / L)
    return Chart2D(tuple(n), J4, hess)


def annulus_chart2d(n, r0):
    """annulus_chart in two dimensions: axis 0 radial (r = r0 + x), axis 1
    around the cylinders (theta = y / r0); g = diag(1, (r / r0)^2)."""
    x, y = grid2d(n)
    r, th = r0 + x, y / r0
    c, s = np.cos(th), np.sin(th)
    J4 = np.stack([c, -(r / r0) * s, s, (r / r0) * c])
    hess = np.zeros((8, x.size))  # d_j d_k h^a at a*4 + j*2 + k
    hess[0 * 4 + 1] = hess[0 * 4 + 2] = -s / r0
    hess[0 * 4 + 3] = -(r / r0 ** 2) * c
    hess[1 * 4 + 1] = hess[1 * 4 + 2] = c / r0
    hess[1 * 4 + 3] = -(r / r0 ** 2) * s
    return Chart2D(tuple(n), J4, hess)


def flag_channel(n=(257, 65), amp=0.05, width=0.15, center=0.35, re=100.0, tau=0.6):
    """2-D flag-like channel: walls at y = 0 and y = H, a parabolic inlet at x
    = 0 (centre-line speed from Re = U H / nu), an outlet at x = n0 - 1, the top
    wall indented by a Gaussian bump d(x) = -amp H exp(-((x - c L)/(w L))^2 / 2)
    (a concavity, the shape of the paper's stability study).  Returns a dict
    with the chart, bcs (1 wall, 2 inflow, 3 outflow) and the inlet velocity
    (contravariant, [2, n1])."""
    x, y = grid2d(n)
    L, H = n[0] - 1, n[1] - 1
    xs = (x - center * L) / (width * L)
    g = np.exp(-0.5 * xs * xs)
    d = -amp * H * g
    dd = amp * H * g * xs / (width * L)
    ddd = amp * H * g * (1.0 - xs * xs) / (width * L) ** 2
    ch = channel_chart2d(n, d, dd, ddd)
    nu = (tau - 0.5) / 3.0
    U = re * nu / H
    yy = np.arange(n[1], dtype=np.float64)
    u_in = np.zeros((2, n[1]))
    u_in[0] = 4.0 * U * yy * (H - yy) / (H * H)  # the inlet column has d = 0 there (J = identity)
    return dict(n=tuple(n), chart=ch, bc_lo=(2, 1), bc_hi=(3, 1), tau=tau, u_in=u_in, umax=U)


def plain_fp64_channel(n=(16, 32, 16), layout=LAYOUT):
    """Static one-mode channel (16 x 16 x 32 nodes, 32 along the flow):
    d = 0.05 H sin(2 pi s / n_flow), tau = 0.8, body force for umax = 0.05."""
    return periodic_channel(n, 0.8, 0.05, 1, 0.05, 0, modes=([1], [0], [-np.pi / 2]),
                            coeffs=[1.0], layout=layout)


def dynamic_channel(n=(128, 256, 128), seed=2000, n_modes=16, amp=0.10, tau=0.6, re=100.0,
                    t=0.0, period=2000.0, kmax=4, lmax=3, layout=LAYOUT):
    """Walls across the wall axis, periodic span, parabolic inflow at the low
    flow face and outflow at the high one; deformation scaled by
    a(t) = sin^2(pi t/period)."""
    nu = (tau - 0.5) / 3.0
    w = layout[0]
    H = n[w] - 1
    umax = re * nu / H
    base = fourier_deformation(n, n_modes, amp, seed, flow_periodic=False, kmax=kmax, lmax=lmax,
                               layout=layout)
    lo, hi = _bcs(layout, INFLOW, OUTFLOW)
    wl = dict(n=tuple(n), bc_lo=lo, bc_hi=hi, tau=tau, fext=(0.0, 0.0, 0.0), base=base, umax=umax,
              period=period, layout=layout, wall_axis=w)
    wl["chart"], wl["faces"] = dynamic_channel_at(wl, t)
    wl["dfm"] = base.scaled(time_law(t, period)[0])
    return wl


def developed_flow(n, umax, seed, layout=LAYOUT):
    """A smooth initial state: the parabolic profile across the wall axis
    along the flow axis everywhere, a 1e-3 density perturbation and a 1 %
    velocity perturbation (seeded), so that relative errors of u are well
    conditioned from the first step."""
    rng = np.random.default_rng(seed)
    w, _, fl = layout
    r = np.stack(grid(n))
    H = n[w] - 1
    u = np.zeros(r.shape)
    u[fl] = 4.0 * umax * r[w] * (H - r[w]) / H ** 2
    ph = rng.uniform(0, 2 * np.pi, size=3)
    bump = sum(np.sin(2 * np.pi * r[a] / n[a] + ph[a]) for a in range(3))
    rho = 1.0 + 1e-3 * bump
    u[fl] *= 1.0 + 0.01 * bump
    return rho, u


def dynamic_channel_at(w, t):
    """The chart and face velocities of a dynamic_channel workload at time t."""
    a, adot = time_law(t, w["period"])
    lay = w["layout"]
    chart = channel_chart(w["n"], w["base"].scaled(a), lay)
    faces = {(lay[2], 0): inflow_profile(w["n"], chart, w["umax"], lay),
             (lay[0], 1): wall_velocity(w["n"], chart, w["base"].scaled(adot), lay)}
    return chart, faces


def max_slope(dfm):
    """Largest wall slope |grad d| of a deformation over the nodes."""
    return float(np.sqrt(dfm.dp ** 2 + dfm.ds ** 2).max())


def batch_channels(nb=64, seed0=4000, side=(32, 96), n_modes=4, amp=(0.02, 0.10), tau=(0.55, 1.0), umax=0.05,
                   layout=LAYOUT, kmax=2, lmax=1, slope_cap=0.25):
    """Independent periodic channels of uneven sizes (walls across the wall
    axis, periodic span and flow, body-force drive with centre-line speed
    umax): channel i draws its three sides from U{side[0]..side[1]}, its
    deformation amplitude (fraction of the height) from U[amp], tau from
    U[tau] with numpy.random.default_rng(seed0 + i + 100000), and its
    n_modes-mode deformation (wavenumbers up to kmax along the flow, lmax
    across) with seed seed0 + i.  A deformation whose largest wall slope
    exceeds slope_cap is scaled down to it: the second-order method on a
    single-mode channel is stable up to a slope of about 0.3 at tau = 0.6 (and
    0.5 at tau = 0.9), and a height-relative amplitude on a channel taller
    than it is long gives steeper walls than that.  The amplitude a channel
    ends with is its 'amp_eff'."""
    out = []
    for i in range(nb):
        rng = np.random.default_rng(seed0 + i + 100000)
        n = tuple(int(v) for v in rng.integers(side[0], side[1] + 1, size=3))
        a = float(rng.uniform(*amp))
        t = float(rng.uniform(*tau))
        w = periodic_channel(n, t, umax, n_modes, a, seed0 + i, layout=layout, kmax=kmax, lmax=lmax)
        s = max_slope(w["dfm"])
        if slope_cap is not None and s > slope_cap:
            a *= slope_cap / s
            w = periodic_channel(n, t, umax, n_modes, a, seed0 + i, layout=layout, kmax=kmax, lmax=lmax)
        w["amp_eff"] = a
        out.append(w)
    return out
