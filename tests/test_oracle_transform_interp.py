"""Pins of the oracle's interpolating chart change (Sec. IV.B, transition
maps): it reduces to the node-wise transform when every new node maps to
itself, shifts the state exactly by whole nodes (also a curved chart moved
with it), reproduces moments that are linear in x, clamps points past a wall
to the wall node, and converges at second order for smooth fields."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

P, W = 0, 1


def grid_psi(n, shift=(0.0, 0.0, 0.0)):
    x, y, z = I.grid(n)
    return np.stack([x + shift[0], y + shift[1], z + shift[2]])


def flat(n):
    ch = I.flat_chart(n)
    return ch.g6, ch.dg18, ch.J9


def test_identity_map_equals_node_wise_transform():
    n = (8, 12, 10)
    w = I.periodic_channel(n, 0.7, 0.05, 3, 0.06, 21, kmax=1, lmax=1)
    ch0 = w["chart"]
    ch1 = I.channel_chart(n, w["dfm"].scaled(1.4), w["layout"])
    runs = []
    for interp in (False, True):
        o = oracle.Lattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(ch0.g6, ch0.dg18)
        o.init()
        o.step(15)
        if interp:
            o.transform_interp(ch1.g6, ch1.dg18, ch0.J9, ch1.J9, grid_psi(n))
        else:
            o.transform(ch1.g6, ch1.dg18, ch0.J9, ch1.J9)
        runs.append((o.f.copy(), o.Fprev.copy()))
    assert np.abs(runs[0][0] - runs[1][0]).max() < 1e-14
    assert np.abs(runs[0][1] - runs[1][1]).max() < 1e-14


def test_whole_node_shift_moves_the_moments():
    n = (10, 8, 6)
    g6, dg18, J9 = flat(n)
    o = oracle.Lattice(n, (P, P, P), (P, P, P), tau=0.8)
    o.set_metric(g6, dg18)
    x, y, z = I.grid(n)
    rho0 = 1.0 + 0.05 * np.sin(2 * np.pi * x / n[0]) * np.cos(2 * np.pi * y / n[1])
    u0 = np.stack([0.02 * np.cos(2 * np.pi * y / n[1]), 0.01 * np.sin(2 * np.pi * z / n[2]), 0.0 * x])
    o.init(rho0, u0)
    o.step(5)
    r0, u0s = o.moments(J9)
    o.transform_interp(g6, dg18, J9, J9, grid_psi(n, (1.0, 0.0, 0.0)))
    r1, u1 = o.moments(J9)
    sh = lambda a: np.roll(a.reshape(a.shape[:-1] + n[::-1]), -1, axis=-1).reshape(a.shape)
    assert np.abs(r1 - sh(r0)).max() < 1e-13
    assert np.abs(u1 - sh(u0s)).max() < 1e-13


def test_moments_linear_in_x_are_interpolated_exactly():
    n = (12, 6, 6)
    g6, dg18, J9 = flat(n)
    lo = (W, P, P)
    o = oracle.Lattice(n, lo, lo, tau=0.8)
    o.set_metric(g6, dg18)
    x, y, z = I.grid(n)
    o.init(1.0 + 0.01 * x, np.stack([0.02 + 0 * x, -0.01 + 0 * x, 0.005 + 0 * x]))
    o.transform_interp(g6, dg18, J9, J9, grid_psi(n, (0.37, 0.0, 0.0)))
    r, u = o.moments(J9)
    inner = (x >= 1) & (x <= n[0] - 3)
    assert np.abs(r[inner] - (1.0 + 0.01 * (x[inner] + 0.37))).max() < 1e-13
    jx = r * u[0]
    # rho u is interpolated; u stays 0.02 where rho u and rho are both linear
    assert np.abs(jx[inner] - 0.02 * (1.0 + 0.01 * (x[inner] + 0.37))).max() < 1e-13


def test_trilinear_interpolation_converges_at_second_order():
    errs = []
    for m in (16, 32, 64):
        n = (m, 4, 4)
        g6, dg18, J9 = flat(n)
        o = oracle.Lattice(n, (P, P, P), (P, P, P), tau=0.8)
        o.set_metric(g6, dg18)
        x, y, z = I.grid(n)
        k = 2 * np.pi / m
        o.init(1.0 + 0.05 * np.sin(k * x), np.zeros((3, x.size)))
        o.transform_interp(g6, dg18, J9, J9, grid_psi(n, (0.5, 0.0, 0.0)))
        r, _ = o.moments(J9)
        ref = 1.0 + 0.05 * np.sin(k * (x + 0.5))
        errs.append(np.abs(r - ref).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), (errs, rates)


def test_whole_node_shift_on_a_curved_chart():
    """A curved chart moved by one node along a periodic axis: the transition
    map is psi(x) = x + e, D phi = J~(x)^-1 J(psi(x)) is the identity, and
    every node takes the density and Cartesian velocity of the old node
    x + e exactly (the old Jacobian is read at psi(x), not at x)."""
    n = (6, 12, 8)
    w = I.periodic_channel(n, 0.7, 0.05, 3, 0.06, 21, kmax=1, lmax=1)
    ch0 = w["chart"]
    roll = lambda a: np.roll(a.reshape(a.shape[:-1] + n[::-1]), -1, axis=-2).reshape(a.shape)  # y -> y + 1
    g6n, dg18n, J9n = roll(ch0.g6), roll(ch0.dg18), roll(ch0.J9)
    assert np.abs(J9n - ch0.J9).max() > 1e-3  # the chart varies along the shift
    o = oracle.Lattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(ch0.g6, ch0.dg18)
    o.init()
    o.step(10)
    r0, v0 = o.moments(ch0.J9)
    o.transform_interp(g6n, dg18n, ch0.J9, J9n, grid_psi(n, (0.0, 1.0, 0.0)))
    r1, v1 = o.moments(J9n)
    assert np.abs(r1 - roll(r0)).max() < 1e-13
    assert np.abs(v1 - roll(v0)).max() < 1e-14
    assert np.abs(v0).max() > 1e-3


def test_points_beyond_a_wall_take_the_wall_node():
    """A transition map that points past a non-periodic face is clamped to
    the face: a node whose old point lies beyond the wall takes the wall
    node's moments (the wall's velocity, here at rest)."""
    n = (12, 6, 6)
    g6, dg18, J9 = flat(n)
    lo = (W, P, P)
    o = oracle.Lattice(n, lo, lo, tau=0.8)
    o.set_metric(g6, dg18)
    x, y, z = I.grid(n)
    o.init(1.0 + 0.01 * x, np.stack([0.02 + 0 * x, 0 * x, 0 * x]))
    o.transform_interp(g6, dg18, J9, J9, grid_psi(n, (1.37, 0.0, 0.0)))
    r, u = o.moments(J9)
    beyond = x == n[0] - 2  # psi = n0 - 0.63 > n0 - 1
    assert np.abs(u[0][beyond]).max() < 1e-15
    assert np.abs(r[beyond] - (1.0 + 0.01 * (n[0] - 2))).max() < 1e-13  # the wall node carries its inner density
    inside = x == n[0] - 3  # psi = n0 - 1.63: between the last fluid node and the wall
    assert np.abs(u[0][inside] - 0.02 * (1 - 0.37) * (1.0 + 0.01 * (n[0] - 2)) / r[inside]).max() < 1e-13
