"""Circular Couette flow (Sec. V.B) through the C ABI: polar coordinates on
the lattice (axis 0 radial between two counter-rotating cylinders with the
paper's radius ratio 1.063, axis 1 around them), FP64 storage, against the
oracle on the same inputs and against the analytic profile."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.late]
P, W = oracle.PERIODIC, oracle.WALL
HERE = os.path.dirname(os.path.abspath(__file__))
CC = json.load(open(os.path.join(HERE, "golden", "paper_bounds.json")))["couette"]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_circular_couette_fp64_against_oracle_and_analytic():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    nx, ny, nz, U, tau = 17, 4, 4, 1e-3, 1.0
    L = nx - 1
    r0 = L / (CC["R2"] / CC["R1"] - 1.0)
    n = (nx, ny, nz)
    ch = I.annulus_chart(n, r0)
    g = CurvedLattice(n, (W, P, P), (W, P, P), tau=tau, storage="fp64")
    g.set_chart(ch)
    o = oracle.Lattice(n, (W, P, P), (W, P, P), tau=tau)
    o.set_metric(ch.g6, ch.dg18)
    om1 = U / r0
    om2 = om1 * CC["Omega2"] / CC["Omega1"]
    R1, R2 = r0, r0 + L
    for side, om, R in ((0, om1, R1), (1, om2, R2)):
        u = np.zeros((3, ny * nz))
        u[1] = om * R * r0 / R  # contravariant: u^1 = v_theta r0 / r
        g.set_boundary_velocity(0, side, u)
        o.set_face_velocity(0, side, u)
    g.init_equilibrium()
    o.init()
    steps = int(4 * L ** 2 / ((tau - 0.5) / 3.0))
    g.step(steps)
    o.step(steps)
    rg, vg = g.moments(cartesian=True)
    ro, vo = o.moments(ch.J9)
    assert rel(rg, ro) < 1e-12 and rel(vg, vo) < 1e-9, (rel(rg, ro), rel(vg, vo))
    x, y, _ = I.grid(n)
    r, th = r0 + x, y / r0
    vt = -np.sin(th) * vg[0] + np.cos(th) * vg[1]
    A = (om2 * R2 ** 2 - om1 * R1 ** 2) / (R2 ** 2 - R1 ** 2)
    B = (om1 - om2) * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    assert rel(vt, A * r + B / r) < 5e-6
