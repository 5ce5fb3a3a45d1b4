"""Circular Couette flow (Sec. V.B, boundary slip): the fluid between two
concentric cylinders of radii R1 < R2 turning at angular velocities Omega1,
Omega2, with the paper's radius ratio R2/R1 = 1.063 and Omega2 = -Omega1
(tests/golden/paper_bounds.json).  The lattice carries polar coordinates:
axis 0 radial, axis 1 around the cylinders, so the metric is curved
(g_11 = (r/r0)^2, Gamma^r_{theta theta} and Gamma^theta_{r theta} nonzero)
and the cylinders are walls moving along their tangent.

The steady azimuthal velocity is the textbook v(r) = A r + B / r with
A = (Omega2 R2^2 - Omega1 R1^2) / (R2^2 - R1^2) and
B = (Omega1 - Omega2) R1^2 R2^2 / (R2^2 - R1^2), the unique solution of the
steady Stokes equations with v(R_k) = Omega_k R_k.  (The printed C2 carries
the opposite sign, which misses both boundary values.)  The oracle converges
to it at second order while the plane (linear) profile it would give
without the curvature terms misses by 1.6-1.8 %.  The speed is kept low
(inner wall 1e-3) so that compressibility, which the analytic solution
leaves out, stays below the discretisation error.
"""
import json
import os

import numpy as np

import oracle
from paper_1803_07822_gb300 import inputs as I

P, W = oracle.PERIODIC, oracle.WALL
HERE = os.path.dirname(os.path.abspath(__file__))
CC = json.load(open(os.path.join(HERE, "golden", "paper_bounds.json")))["couette"]


def circular_couette(nx, U=1e-3, tau=1.0, ny=4):
    """Gap of nx nodes (walls on the cylinders), ny nodes around (the flow
    does not depend on theta); returns (relative L2 error of v_theta,
    largest |v_r|, relative L2 distance of the linear profile)."""
    L = nx - 1
    ratio = CC["R2"] / CC["R1"]
    r0 = L / (ratio - 1.0)  # inner radius in lattice units
    n = (nx, ny, 1)
    nu = (tau - 0.5) / 3.0
    ch = I.annulus_chart(n, r0)
    lat = oracle.Lattice(n, (W, P, P), (W, P, P), tau=tau)
    lat.set_metric(ch.g6, ch.dg18)
    om1 = U / r0
    om2 = om1 * CC["Omega2"] / CC["Omega1"]
    R1, R2 = r0, r0 + L
    # contravariant velocity around the cylinders: u^1 = v_theta r0 / r
    for side, om, R in ((0, om1, R1), (1, om2, R2)):
        u = np.zeros((3, ny))
        u[1] = om * R * r0 / R
        lat.set_face_velocity(0, side, u)
    lat.init()
    lat.step(int(4 * L ** 2 / nu))
    _, v = lat.moments(ch.J9)
    x, y, _ = I.grid(n)
    r, th = r0 + x, y / r0
    vt = -np.sin(th) * v[0] + np.cos(th) * v[1]
    vr = np.cos(th) * v[0] + np.sin(th) * v[1]
    A = (om2 * R2 ** 2 - om1 * R1 ** 2) / (R2 ** 2 - R1 ** 2)
    B = (om1 - om2) * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    exact = A * r + B / r
    linear = om1 * R1 + (om2 * R2 - om1 * R1) * x / L
    nrm = np.linalg.norm(exact)
    return np.linalg.norm(vt - exact) / nrm, np.abs(vr).max(), np.linalg.norm(linear - exact) / nrm


def test_analytic_profile_meets_the_walls():
    R1, R2, o1, o2 = CC["R1"], CC["R2"], CC["Omega1"], CC["Omega2"]
    A = (o2 * R2 ** 2 - o1 * R1 ** 2) / (R2 ** 2 - R1 ** 2)
    B = (o1 - o2) * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    assert abs(A * R1 + B / R1 - o1 * R1) < 1e-18 and abs(A * R2 + B / R2 - o2 * R2) < 1e-18


def test_circular_couette_second_order():
    res = [circular_couette(m) for m in (9, 17, 33)]
    errs = np.array([e for e, _, _ in res])
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[0] < 2e-5 and np.all(rates > 1.9), (errs, rates)
    for e, vr, lin in res:
        assert vr < 1e-3 * 1e-3 * 0.1  # no radial flow: |v_r| < 1e-4 of the wall speed
        assert lin > 500 * e  # the curvature terms are what the profile resolves
