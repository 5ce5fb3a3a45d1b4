"""Pins of the two-dimensional (D2Q9) oracle against what the method fixes:
the flat metric reduces it to textbook D2Q9 BGK; rest stays at rest and mass
is conserved; plane Poiseuille flow between walls on the nodes; the same flow
under a re-parametrised (curved) metric converges to the analytic Cartesian
profile; the wall force at rest is pressure times length; a chart change to
the same chart leaves the moments; the boundary nodes carry the fields their
rules define."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

P, W = 0, 1


def textbook_d2q9(f, tau, steps, n):
    """Plain D2Q9 BGK, periodic, pull streaming: f_eq = w rho (1 + 3 c.u +
    9/2 (c.u)^2 - 3/2 u^2)."""
    c, w = oracle.lattice2d()
    f = f.reshape(9, n[1], n[0]).copy()
    for _ in range(steps):
        rho = f.sum(0)
        u = np.einsum("la,lyx->ayx", c.astype(float), f) / rho
        cu = np.einsum("la,ayx->lyx", c.astype(float), u)
        feq = w[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u * u).sum(0))
        fs = f - (f - feq) / tau
        f = np.stack([np.roll(np.roll(fs[l], c[l, 1], axis=0), c[l, 0], axis=1) for l in range(9)])
    return f.reshape(9, -1)


def test_flat_periodic_is_textbook_bgk():
    n = (12, 10)
    x, y = I.grid2d(n)
    rho0 = 1.0 + 0.02 * np.sin(2 * np.pi * x / n[0])
    u0 = np.stack([0.03 * np.cos(2 * np.pi * y / n[1]), 0.01 * np.sin(2 * np.pi * x / n[0])])
    o = oracle.Lattice2D(n, (P, P), (P, P), tau=0.7)
    ch = I.flat_chart2d(n)
    o.set_metric(ch.g3, ch.dg6)
    o.init(rho0, u0)
    f0 = o.f.copy()
    o.step(40)
    ref = textbook_d2q9(f0, 0.7, 40, n)
    assert np.abs(o.f - ref).max() < 1e-13


def test_rest_and_mass():
    n = (9, 7)
    ch = I.flat_chart2d(n)
    o = oracle.Lattice2D(n, (P, W), (P, W), tau=0.8)
    o.set_metric(ch.g3, ch.dg6)
    o.init()
    m0 = o.mass()
    o.step(50)
    r, u = o.moments()
    assert np.abs(u).max() < 1e-15 and np.abs(r - 1).max() < 1e-14
    x, y = I.grid2d((8, 8))
    o = oracle.Lattice2D((8, 8), (P, P), (P, P), tau=0.8)
    ch = I.flat_chart2d((8, 8))
    o.set_metric(ch.g3, ch.dg6)
    o.init(1 + 0.05 * np.cos(2 * np.pi * x / 8), np.stack([0.02 + 0 * x, 0 * x]))
    m0 = o.mass()
    o.step(100)
    assert abs(o.mass() - m0) < 1e-12 * m0


def poiseuille(n1, eps, tau=1.0, umax=0.02):
    """Plane Poiseuille flow between walls on the nodes y = 0, L (L = n1 - 1),
    driven by F = 8 nu umax / L^2 along x, under the chart y_c = y + eps (L/pi)
    sin(pi y/L); relative L2 error of the Cartesian velocity at the nodes'
    positions against F y_c (L - y_c) / (2 nu rho)."""
    n = (4, n1)
    L = n1 - 1
    nu = (tau - 0.5) / 3.0
    F = 8.0 * nu * umax / L ** 2
    ch = I.reparam_chart2d(n, eps)
    o = oracle.Lattice2D(n, (P, W), (P, W), tau=tau, fext=(F, 0.0))
    o.set_metric(ch.g3, ch.dg6)
    o.init()
    o.step(int(6 * L ** 2 / nu))
    r, v = o.moments(ch.J4)
    y = I.grid2d(n)[1]
    yc = y + eps * (L / np.pi) * np.sin(np.pi * y / L)
    exact = F * yc * (L - yc) / (2.0 * nu * r.mean())
    return np.linalg.norm(v[0] - exact) / np.linalg.norm(exact), v


def test_flat_poiseuille_matches_analytic():
    err, v = poiseuille(17, 0.0)
    assert err < 1e-3
    assert np.abs(v[1]).max() < 1e-14


def test_reparametrised_poiseuille_converges_at_second_order():
    errs = [poiseuille(n1, 0.1)[0] for n1 in (9, 17, 33)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.7), (errs, rates)


def test_wall_force_at_rest_is_pressure_times_length():
    n = (10, 8)
    for ch in (I.flat_chart2d(n), I.channel_chart2d(n, *[np.full(80, v) for v in (0.3, 0.0, 0.0)])):
        o = oracle.Lattice2D(n, (P, W), (P, W), tau=0.8)
        o.set_metric(ch.g3, ch.dg6)
        o.init()
        F = o.wall_force(1, 1, ch.J4)
        assert abs(F[1] - n[0] / 3.0) < 1e-12 and abs(F[0]) < 1e-14


def test_transform_to_the_same_chart_keeps_the_moments():
    w = I.flag_channel((40, 17), amp=0.05)
    ch = w["chart"]
    o = oracle.Lattice2D(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"])
    o.set_metric(ch.g3, ch.dg6)
    o.set_face_velocity(0, 0, w["u_in"])
    o.init()
    o.step(30)
    r0, u0 = o.moments(ch.J4)
    o.transform(ch.g3, ch.dg6, ch.J4, ch.J4)
    r1, u1 = o.moments(ch.J4)
    assert np.abs(r1 - r0).max() < 1e-14 and np.abs(u1 - u0).max() < 1e-14


def _boundary_rule2(n, bc_lo, bc_hi, r):
    prio = {1: 3, 2: 2, 3: 1}
    best, inner = None, list(r)
    for a in range(2):
        for s, bc in ((0, bc_lo[a]), (1, bc_hi[a])):
            if bc == P or r[a] != (0 if s == 0 else n[a] - 1):
                continue
            inner[a] = r[a] + (1 if s == 0 else -1)
            if best is None or prio[bc] > prio[best[0]]:
                best = (bc, a, s)
    return None if best is None else (*best, tuple(inner))


@pytest.mark.parametrize("bcs", [((2, 1), (3, 1)), ((2, 2), (3, 3)), ((3, 2), (1, 3))])
def test_boundary_fields_on_every_boundary_node(bcs):
    """What the boundary rules mean, on a curved state after a few steps: a
    wall or inflow node carries the inner node's density and the imposed
    contravariant velocity, an outflow node the inner node's density and
    velocity; the inner node is one step inward along every non-periodic face
    of the node, and the rule is the one of highest priority (wall > inflow >
    outflow, then the lower axis, then the low side)."""
    bc_lo, bc_hi = bcs
    w = I.flag_channel((11, 9), amp=0.05, tau=0.8)
    n = w["n"]
    rng = np.random.default_rng(5)
    faces = {}
    o = oracle.Lattice2D(n, bc_lo, bc_hi, tau=0.8)
    o.set_metric(w["chart"].g3, w["chart"].dg6)
    for a in range(2):
        for s, bc in ((0, bc_lo[a]), (1, bc_hi[a])):
            if bc in (1, 2):
                faces[(a, s)] = 0.01 * rng.standard_normal((2, n[1 - a]))
                o.set_face_velocity(a, s, faces[(a, s)])
    o.init()
    o.step(10)
    rho, u = o.moments()
    seen = set()
    for y in range(n[1]):
        for x in range(n[0]):
            rule = _boundary_rule2(n, bc_lo, bc_hi, (x, y))
            if rule is None:
                continue
            bc, a, s, inner = rule
            v, vi = x + n[0] * y, inner[0] + n[0] * inner[1]
            seen.add(bc)
            assert abs(rho[v] - rho[vi]) < 1e-13 * rho[vi]
            want = u[:, vi] if bc == 3 else faces[(a, s)][:, (x, y)[1 - a]]
            assert np.abs(u[:, v] - want).max() < 1e-14, ((x, y), bc)
    assert seen == {bc for bc in bc_lo + bc_hi if bc}


def test_circular_couette_second_order():
    """Circular Couette flow (Sec. V.B) on polar lattice coordinates: the
    radius ratio 1.063 and Omega2 = -Omega1 of the paper, inner wall speed
    1e-3; the Cartesian azimuthal profile converges at second order to
    A r + B / r (B = (Omega1 - Omega2) R1^2 R2^2 / (R2^2 - R1^2))."""
    errs = []
    for m in (9, 17, 33):
        L = m - 1
        r0 = L / 0.063
        n = (m, 4)
        ch = I.annulus_chart2d(n, r0)
        o = oracle.Lattice2D(n, (W, P), (W, P), tau=1.0)
        o.set_metric(ch.g3, ch.dg6)
        om1 = 1e-3 / r0
        om2 = -om1
        R1, R2 = r0, r0 + L
        for side, om in ((0, om1), (1, om2)):
            o.set_face_velocity(0, side, np.stack([np.zeros(4), np.full(4, om * r0)]))  # u^1 = v_theta r0 / r
        o.init()
        o.step(int(4 * L ** 2 * 6))
        _, v = o.moments(ch.J4)
        x, y = I.grid2d(n)
        r, th = r0 + x, y / r0
        vt = -np.sin(th) * v[0] + np.cos(th) * v[1]
        A = (om2 * R2 ** 2 - om1 * R1 ** 2) / (R2 ** 2 - R1 ** 2)
        B = (om1 - om2) * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
        ex = A * r + B / r
        errs.append(np.linalg.norm(vt - ex) / np.linalg.norm(ex))
        lin = om1 * R1 + (om2 * R2 - om1 * R1) * x / L
        assert np.linalg.norm(lin - ex) / np.linalg.norm(ex) > 500 * errs[-1]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[0] < 2e-5 and np.all(rates > 1.9), (errs, rates)


def test_flat_couette_wall_force_is_the_exact_stress():
    """Plane Couette flow between walls on the nodes y = 0 (at rest) and
    y = L (moving at U along x): at steady state the force of the fluid on
    each wall is the exact shear rho nu U / L per wall node (forward on the
    resting wall, backward on the moving one) and the pressure rho theta
    normal to it."""
    for n1, tau in ((9, 1.0), (13, 0.7)):
        n = (4, n1)
        L = n1 - 1
        nu = (tau - 0.5) / 3.0
        U = 0.05
        ch = I.flat_chart2d(n)
        o = oracle.Lattice2D(n, (P, W), (P, W), tau=tau)
        o.set_metric(ch.g3, ch.dg6)
        o.set_face_velocity(1, 1, np.stack([np.full(4, U), np.zeros(4)]))
        o.init()
        o.step(int(6 * L ** 2 / nu))
        rho, _ = o.moments()
        F0, F1 = o.wall_force(1, 0, ch.J4), o.wall_force(1, 1, ch.J4)
        shear = 4 * rho.mean() * nu * U / L
        assert abs(F0[0] - shear) < 1e-12 * shear and abs(F1[0] + shear) < 1e-12 * shear, (F0, F1, shear)
        assert abs(F0[1] + 4 * rho.mean() / 3) < 1e-11 and abs(F1[1] - 4 * rho.mean() / 3) < 1e-11


def test_forcing_recomposition_moments_2d():
    """The recomposed forcing carries the moments it is built from (Eq.
    forcing2 in 2-D): sum F sqrt(g) = A, sum F c sqrt(g) = B, sum F c c
    sqrt(g) = C, for random moments and sqrt(g) (the fourth moment of the
    D2Q9 weights is isotropic)."""
    c, w = oracle.lattice2d()
    c = c.astype(float)
    rng = np.random.default_rng(21)
    for _ in range(5):
        A = rng.standard_normal()
        B = rng.standard_normal(2)
        C = rng.standard_normal((2, 2))
        C = C + C.T
        sg = rng.uniform(0.7, 1.3)
        F = oracle.forcing_recompose2d(A, B, C.ravel(), sg)
        assert abs((F * sg).sum() - A) < 1e-13
        assert np.abs(np.einsum("l,la->a", F * sg, c) - B).max() < 1e-13
        assert np.abs(np.einsum("l,la,lb->ab", F * sg, c, c) - C).max() < 1e-13


def test_mass_at_rest_is_the_area_of_the_chart():
    """At rest (rho = 1) the mass sum sqrt(g) rho is the sum over the nodes of
    |det J|, the area each node stands for in Cartesian space."""
    w = I.flag_channel((40, 17), amp=0.08)
    ch = w["chart"]
    o = oracle.Lattice2D(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"])
    o.set_metric(ch.g3, ch.dg6)
    o.init()
    detJ = np.abs(ch.J4[0] * ch.J4[3] - ch.J4[1] * ch.J4[2])
    assert abs(o.mass() - detJ.sum()) < 1e-12 * detJ.sum()
    assert abs(detJ.sum() - detJ.size) > 1e-3 * detJ.size  # the chart is not area-preserving


def test_chart_change_keeps_density_and_cartesian_velocity():
    """The node-wise chart change maps u to J~^-1 J u (Sec. IV.B), so every
    fluid node keeps its density and its Cartesian velocity through a change
    between two different charts."""
    w0 = I.flag_channel((40, 17), amp=0.05)
    w1 = I.flag_channel((40, 17), amp=0.09, center=0.5)
    c0, c1 = w0["chart"], w1["chart"]
    n = w0["n"]
    rng = np.random.default_rng(8)
    N = n[0] * n[1]
    rho0 = 1.0 + 0.01 * rng.standard_normal(N)
    u0 = 0.02 * rng.standard_normal((2, N))
    o = oracle.Lattice2D(n, (P, W), (P, W), tau=0.8)
    o.set_metric(c0.g3, c0.dg6)
    o.init(rho0, u0)
    r0, v0 = o.moments(c0.J4)
    o.transform(c1.g3, c1.dg6, c0.J4, c1.J4)
    r1, v1 = o.moments(c1.J4)
    y = I.grid2d(n)[1]
    fluid = (y > 0) & (y < n[1] - 1)
    assert np.abs(r1 - r0)[fluid].max() < 1e-13
    assert np.abs(v1 - v0)[:, fluid].max() < 1e-14
    assert np.abs(c1.J4 - c0.J4).max() > 0.01  # the charts differ


def test_forcing_C_parallel_field_has_no_theta_part_2d():
    """As in three dimensions: a uniform Cartesian flow in polar coordinates
    is a parallel field (nabla_k j^i = d_k j^i + Gamma^i_kl j^l = 0), so the
    theta part of C^ij (Eq. forcing-C) vanishes and C does not depend on theta;
    without the Gamma rho u term it would."""
    n = (7, 9)
    ch = I.annulus_chart2d(n, 5.0)
    N = int(np.prod(n))
    sg, gi, gam = oracle.geometry2d(n, ch.g3, ch.dg6)
    J = np.moveaxis(ch.J4.reshape(2, 2, N), 2, 0)
    Jinv = np.linalg.inv(J)
    dJ = np.moveaxis(ch.hess.reshape(2, 2, 2, N), 3, 0)  # [n, b, m, k] = d_k J^b_m
    rng = np.random.default_rng(22)
    worst, scale = 0.0, 0.0
    for v in rng.choice(N, size=10, replace=False):
        j = Jinv[v] @ (0.05 * rng.standard_normal(2))
        Dj = -np.einsum("ib,bmk,m->ki", Jinv[v], dJ[v], j)
        T = rng.standard_normal((2, 2))
        T = T + T.T
        C = [oracle.forcing_moments2d(j, T.ravel(), Dj.ravel(), gi[:, v], gam[:, v], th)[2] for th in (1 / 3, 0.25)]
        C0 = [oracle.forcing_moments2d(j, T.ravel(), Dj.ravel(), gi[:, v], np.zeros(8), th)[2] for th in (1 / 3, 0.25)]
        worst = max(worst, np.abs(C[0] - C[1]).max())
        scale = max(scale, np.abs(C0[0] - C0[1]).max())
    assert scale > 1e-4
    assert worst < 1e-15 + 1e-12 * scale, (worst, scale)
