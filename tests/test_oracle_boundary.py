"""Pins of the oracle's boundary rules (walls and inflow: non-equilibrium
extrapolation with the velocity imposed on the boundary node; outflow: zero
gradient).

What the rules mean fixes the macroscopic fields on the boundary nodes of any
state under any metric: a wall or inflow node carries the inner node's density
and the imposed (contravariant) velocity; an outflow node carries the inner
node's density and momentum.  The inner node is one step inward along every
non-periodic face the node lies on, and a node on several faces takes the rule
of the face of highest priority (wall > inflow > outflow, then the lower axis,
then the low side).  Checked on every boundary node of curved, moving states.

Plane Couette flow, whose steady profile is linear between the walls on the
nodes, pins the moving wall:

- flat metric: the linear profile is an exact steady state of BGK with this
  wall rule, so it is reached to rounding (3-D and 2-D);
- a uniform stretch of the axis along which the wall moves: the wall velocity
  is contravariant, u^z = U / s, and the Cartesian profile is still exact
  (treating it as Cartesian gives an O(s - 1) error);
- the wall-normal re-parametrisation x_c = x + eps (L/pi) sin(pi x/L): the
  Cartesian profile at the nodes' positions converges at second order
  (Sec. V.A validates the method by second-order convergence).
"""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

P, W, IN, OUT = oracle.PERIODIC, oracle.WALL, oracle.INFLOW, oracle.OUTFLOW
U = 0.05
PRIORITY = {W: 3, IN: 2, OUT: 1}


def boundary_rule(n, bc_lo, bc_hi, r):
    """(rule, axis, side, inner node) of node r, or None for a fluid node."""
    best, inner = None, list(r)
    for a in range(3):
        for s, bc in ((0, bc_lo[a]), (1, bc_hi[a])):
            if bc == P or r[a] != (0 if s == 0 else n[a] - 1):
                continue
            inner[a] = r[a] + (1 if s == 0 else -1)
            if best is None or PRIORITY[bc] > PRIORITY[best[0]]:
                best = (bc, a, s)
    return None if best is None else (*best, tuple(inner))


def check_boundary_fields(n, bc_lo, bc_hi, ch, faces, steps):
    lat = oracle.Lattice(n, bc_lo, bc_hi, tau=0.8)
    lat.set_metric(ch.g6, ch.dg18)
    for (a, s), u in faces.items():
        lat.set_face_velocity(a, s, u)
    lat.init()
    lat.step(steps)
    fb = lat.filled()
    assert np.isfinite(fb).all()
    c, _ = oracle.lattice()
    rho = (fb * lat.sqrtg).sum(0)
    j = np.einsum("la,ln->an", c.astype(float), fb * lat.sqrtg)
    node = lambda r: r[0] + n[0] * (r[1] + n[1] * r[2])
    seen = {W: 0, IN: 0, OUT: 0}
    for z in range(n[2]):
        for y in range(n[1]):
            for x in range(n[0]):
                rule = boundary_rule(n, bc_lo, bc_hi, (x, y, z))
                if rule is None:
                    continue
                bc, a, s, inner = rule
                v, vi = node((x, y, z)), node(inner)
                seen[bc] += 1
                assert abs(rho[v] - rho[vi]) < 1e-13 * rho[vi]
                if bc == OUT:
                    assert np.abs(j[:, v] - j[:, vi]).max() < 1e-14
                    continue
                r = (x, y, z)
                o = sorted(((a + 1) % 3, (a + 2) % 3))
                u = faces[(a, s)][:, r[o[0]] + n[o[0]] * r[o[1]]] if (a, s) in faces else np.zeros(3)
                assert np.abs(j[:, v] / rho[v] - u).max() < 1e-14, (r, bc, a, s)
    return seen


def test_boundary_fields_dynamic_channel():
    """Walls across z (the top one moving), inflow at the low flow face with
    the parabolic profile, outflow at the high one, a curved chart."""
    w = I.dynamic_channel(n=(6, 10, 7), t=500.0)
    seen = check_boundary_fields(w["n"], w["bc_lo"], w["bc_hi"], w["chart"], w["faces"], 12)
    assert min(seen.values()) > 0


def test_boundary_fields_mixed_faces_and_priorities():
    """Inflow on two faces and outflow on two (edges where the rules meet and
    ties between faces of one rule), walls across z, random face velocities."""
    w = I.dynamic_channel(n=(6, 10, 7), t=500.0)
    n = w["n"]
    lo, hi = (IN, IN, W), (OUT, OUT, W)
    rng = np.random.default_rng(11)
    faces = {(0, 0): 0.01 * rng.standard_normal((3, n[1] * n[2])),
             (1, 0): 0.01 * rng.standard_normal((3, n[0] * n[2])),
             (2, 1): 0.01 * rng.standard_normal((3, n[0] * n[1]))}
    seen = check_boundary_fields(n, lo, hi, w["chart"], faces, 8)
    assert min(seen.values()) > 0


def couette3d(nx, eps=0.0, s=1.0, tau=1.0, u_wall=None):
    """Walls at x = 0 and x = L (L = nx - 1), the high wall moving along z;
    steady-state Cartesian velocity and density."""
    n = (nx, 1, 1)
    L = nx - 1
    nu = (tau - 0.5) / 3.0
    base = I.reparam_chart(n, eps)
    J9 = base.J9.copy()
    J9[8] = s
    ch = I.Chart(n, J9, base.hess)
    lat = oracle.Lattice(n, (W, P, P), (W, P, P), tau=tau)
    lat.set_metric(ch.g6, ch.dg18)
    lat.set_face_velocity(0, 1, np.array([[0.0], [0.0], [U / s if u_wall is None else u_wall]]))
    lat.init()
    lat.step(int(4 * L ** 2 / nu))  # slowest mode decays as exp(-nu pi^2 t / L^2)
    rho, v = lat.moments(ch.J9)
    exact = U * I.reparam_position(n, eps) / L
    return np.linalg.norm(v[2] - exact) / np.linalg.norm(exact), v, rho


def couette2d(ny, eps=0.0, s=1.0, tau=1.0):
    """Walls at y = 0 and y = L, the high wall moving along x."""
    n = (4, ny)
    L = ny - 1
    nu = (tau - 0.5) / 3.0
    base = I.reparam_chart2d(n, eps)
    J4 = base.J4.copy()
    J4[0] = s
    ch = I.Chart2D(n, J4, base.hess)
    lat = oracle.Lattice2D(n, (P, W), (P, W), tau=tau)
    lat.set_metric(ch.g3, ch.dg6)
    lat.set_face_velocity(1, 1, np.stack([np.full(n[0], U / s), np.zeros(n[0])]))
    lat.init()
    lat.step(int(4 * L ** 2 / nu))
    rho, v = lat.moments(ch.J4)
    y = I.grid2d(n)[1]
    exact = U * (y + eps * (L / np.pi) * np.sin(np.pi * y / L)) / L
    return np.linalg.norm(v[0] - exact) / np.linalg.norm(exact), v, rho


@pytest.mark.parametrize("nx", [9, 17])
def test_flat_couette_is_exact(nx):
    err, v, rho = couette3d(nx)
    assert err < 1e-12 and np.abs(v[:2]).max() < 1e-14 and np.abs(rho - 1).max() < 1e-11
    err, v, rho = couette2d(nx)
    assert err < 1e-12 and np.abs(v[1]).max() < 1e-14 and np.abs(rho - 1).max() < 1e-11


def test_wall_velocity_is_contravariant():
    err, _, _ = couette3d(9, s=1.7)
    assert err < 1e-12
    err, _, _ = couette2d(9, s=1.7)
    assert err < 1e-12
    # the same number read as a Cartesian velocity misses by the stretch
    err, _, _ = couette3d(9, s=1.7, u_wall=U)
    assert err > 0.5


def test_reparametrised_couette_second_order():
    sizes = (17, 33, 65)
    for run in (couette3d, couette2d):
        errs = np.array([run(m, eps=0.1)[0] for m in sizes])
        rates = np.log2(errs[:-1] / errs[1:])
        assert errs[0] < 2e-3 and np.all(rates > 1.8), (run.__name__, errs, rates)


@pytest.mark.parametrize("nx,tau", [(9, 1.0), (17, 0.7), (12, 1.4)])
def test_flat_couette_wall_force_is_the_exact_stress(nx, tau):
    """Momentum transfer on the nodes (Sec. IV.A) in a flowing state: at
    steady plane Couette flow the force of the fluid on each wall is the
    exact viscous shear rho nu U / L (forward on the resting wall, backward
    on the moving one) plus the pressure rho theta normal to the wall, per
    wall node.  Exercises the non-equilibrium part of T (factor 1 - 1/2tau),
    which the rest-state test cannot see."""
    n = (nx, 1, 1)
    L = nx - 1
    nu = (tau - 0.5) / 3.0
    ch = I.flat_chart(n)
    lat = oracle.Lattice(n, (W, P, P), (W, P, P), tau=tau)
    lat.set_metric(ch.g6, ch.dg18)
    lat.set_face_velocity(0, 1, np.array([[0.0], [0.0], [U]]))
    lat.init()
    lat.step(int(6 * L ** 2 / nu))
    rho, _ = lat.moments()
    F0, F1 = lat.wall_force(0, 0, ch.J9), lat.wall_force(0, 1, ch.J9)
    shear = rho.mean() * nu * U / L
    assert abs(F0[2] - shear) < 1e-12 * shear and abs(F1[2] + shear) < 1e-12 * shear
    assert abs(F0[0] + rho[0] / 3.0) < 1e-12 and abs(F1[0] - rho[-1] / 3.0) < 1e-12
    assert abs(F0[1]) < 1e-15 and abs(F1[1]) < 1e-15
