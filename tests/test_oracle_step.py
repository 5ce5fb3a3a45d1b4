"""Whole-step pins of the FP64 oracle.

- flat metric: the method collapses to textbook D3Q19 BGK with forcing
  w c.F/c_s^2 (coded here separately, in numpy);
- rest stays at rest; mass is conserved (exactly when flat and periodic,
  within the paper's 0.1 % under a curved metric);
- Poiseuille flow: analytic profile, second-order convergence of the
  Cartesian velocity under a stretched chart (Sec. V.A);
- momentum transfer on the nodes at rest equals pressure times the
  Cartesian area vector of the wall (Sec. IV.A force coupling);
- the chart-change transformation maps equilibria to equilibria, is a
  projection, and round-trips (Sec. IV.B).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
BOUNDS = json.load(open(os.path.join(HERE, "golden", "paper_bounds.json")))
P, W = oracle.PERIODIC, oracle.WALL
CS2_ = 1.0 / 3.0


def textbook_bgk(f0, n, tau, fext, steps):
    """Standard D3Q19 BGK with the forcing term w c.F / c_s^2 and u = sum f c / rho."""
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                  [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = f0.reshape(19, n[2], n[1], n[0]).copy()
    force = w * (c @ np.asarray(fext)) * 3.0
    for _ in range(steps):
        rho = f.sum(0)
        u = np.einsum("lzyx,la->azyx", f, c) / rho
        cu = np.einsum("la,azyx->lzyx", c, u)
        feq = w[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u ** 2).sum(0))
        fs = f - (f - feq) / tau + force[:, None, None, None]
        for l in range(19):
            fs[l] = np.roll(fs[l], shift=(c[l, 2], c[l, 1], c[l, 0]), axis=(0, 1, 2))
        f = fs
    return f.reshape(19, -1)


def test_flat_periodic_is_textbook_bgk():
    n = (6, 5, 7)
    rng = np.random.default_rng(0)
    N = int(np.prod(n))
    rho0 = 1.0 + 0.05 * rng.standard_normal(N)
    u0 = 0.05 * rng.standard_normal((3, N))
    fext = (1e-4, -2e-4, 3e-4)
    L = oracle.Lattice(n, (P, P, P), tau=0.7, fext=fext)
    L.init(rho0, u0)
    f0 = L.f.copy()
    L.step(20)
    ref = textbook_bgk(f0, n, 0.7, fext, 20)
    assert np.abs(L.f - ref).max() < 1e-13


def test_flat_rest_stays_at_rest_and_mass_exact():
    n = (7, 4, 5)
    L = oracle.Lattice(n, (W, P, P), (W, P, P), tau=0.9)
    L.init()
    m0 = L.mass()
    L.step(200)
    rho, u = L.moments()
    assert np.abs(u).max() < 1e-14 and np.abs(rho - 1).max() < 1e-13
    assert abs(L.mass() - m0) / m0 < 1e-13


def test_flat_periodic_mass_exact_with_flow():
    n = (6, 6, 6)
    rng = np.random.default_rng(4)
    N = int(np.prod(n))
    L = oracle.Lattice(n, (P, P, P), tau=0.6, fext=(0, 0, 1e-4))
    L.init(1 + 0.02 * rng.standard_normal(N), 0.03 * rng.standard_normal((3, N)))
    m0 = L.mass()
    L.step(100)
    assert abs(L.mass() - m0) / m0 < 1e-12


def test_curved_channel_mass_within_paper_bound():
    """Curved static metric with walls and a body force (the 16x16x32 channel,
    one mode, 5 % amplitude): sqrt(g)-weighted mass drift after 1000 steps
    stays within the 0.1 % of the paper's piston test."""
    w = I.plain_fp64_channel()
    L = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    L.set_metric(w["chart"].g6, w["chart"].dg18)
    L.init()
    m0 = L.mass()
    L.step(1000)
    drift = abs(L.mass() - m0) / m0
    assert drift < BOUNDS["mass_rel_drift_max"]["value"]
    rho, u = L.moments(w["chart"].J9)
    assert np.isfinite(u).all() and np.abs(u).max() < 0.1


def _poiseuille(nx, eps, tau=1.0, umax=0.02):
    n = (nx, 1, 1)
    L_ = nx - 1
    nu = (tau - 0.5) / 3.0
    F = 8.0 * nu * umax / L_ ** 2
    ch = I.reparam_chart(n, eps)
    lat = oracle.Lattice(n, (W, P, P), (W, P, P), tau=tau, fext=(0.0, 0.0, F))
    lat.set_metric(ch.g6, ch.dg18)
    lat.init()
    lat.step(int(6 * L_ ** 2 / nu))
    rho, v = lat.moments(ch.J9)
    xc = I.reparam_position(n, eps)
    exact = F * xc * (L_ - xc) / (2.0 * nu * rho.mean())
    return np.linalg.norm(v[2] - exact) / np.linalg.norm(exact), v


def test_poiseuille_flat_matches_analytic():
    err, v = _poiseuille(17, 0.0)
    assert err < 1e-3
    assert np.abs(v[0]).max() < 1e-14 and np.abs(v[1]).max() < 1e-14


def test_poiseuille_stretched_chart_second_order():
    """Cartesian profile under the stretched chart x_c = x + eps L/pi sin(pi x/L)
    (eps = 0.1) converges to the analytic Poiseuille solution at 2nd order."""
    sizes = (9, 17, 33)
    errs = [_poiseuille(nx, 0.1)[0] for nx in sizes]
    slope = np.polyfit(np.log([s - 1 for s in sizes]), np.log(errs), 1)[0]
    assert errs[0] < 0.05
    assert slope < -1.8, (errs, slope)


def test_rest_wall_force_is_pressure_times_area():
    """At rest with uniform rho, T = rho theta g^-1 on the wall nodes, so the
    force on a wall is p * sum (e_j x e_k) over its nodes (the Cartesian area
    vector of the deformed wall, from the chart's tangent vectors)."""
    n = (8, 12, 9)
    dfm = I.fourier_deformation(n, 4, 0.08, seed=21, flow_periodic=True)
    ch = I.channel_chart(n, dfm)
    L = oracle.Lattice(n, (P, P, W), (P, P, W), tau=0.8)
    L.set_metric(ch.g6, ch.dg18)
    L.init()
    J = ch.J9.reshape(3, 3, -1)
    p = 1.0 / 3.0
    for side in (0, 1):
        nodes = I.face_nodes(n, 2, side)
        area = np.cross(J[:, 0, nodes].T, J[:, 1, nodes].T).sum(0)
        F = L.wall_force(2, side, ch.J9)
        s = 1.0 if side else -1.0
        assert np.allclose(F, s * p * area, rtol=0, atol=1e-12)


def test_transform_equilibrium_to_equilibrium_and_round_trip():
    n = (5, 4, 6)
    N = int(np.prod(n))
    rng = np.random.default_rng(8)
    ch1 = I.channel_chart(n, I.fourier_deformation(n, 3, 0.08, 31, flow_periodic=True))
    ch2 = I.channel_chart(n, I.fourier_deformation(n, 3, 0.08, 32, flow_periodic=True))
    rho0 = 1 + 0.05 * rng.standard_normal(N)
    u0 = 0.05 * rng.standard_normal((3, N))
    L = oracle.Lattice(n, (P, P, P), tau=0.8)
    L.set_metric(ch1.g6, ch1.dg18)
    L.init(rho0, u0)
    f1 = L.f.copy()
    L.transform(ch2.g6, ch2.dg18, ch1.J9, ch2.J9)
    # equilibrium maps to the equilibrium of the transformed velocity
    J1 = np.moveaxis(ch1.J9.reshape(3, 3, N), 2, 0)
    J2 = np.moveaxis(ch2.J9.reshape(3, 3, N), 2, 0)
    D = np.linalg.solve(J2, J1)
    u2 = np.einsum("nij,jn->in", D, u0)
    sg2, gi2, _ = oracle.geometry(n, ch2.g6, ch2.dg18)
    for v in range(0, N, 7):
        ref = oracle.feq(rho0[v], rho0[v] * u2[:, v], gi2[:, v], sg2[v])
        assert np.abs(L.f[:, v] - ref).max() < 1e-14
    # and back
    L.transform(ch1.g6, ch1.dg18, ch2.J9, ch1.J9)
    assert np.abs(L.f - f1).max() < 1e-14


def test_transform_is_projection_and_keeps_moments():
    n = (5, 4, 6)
    N = int(np.prod(n))
    rng = np.random.default_rng(9)
    ch1 = I.channel_chart(n, I.fourier_deformation(n, 2, 0.03, 41, True, kmax=1, lmax=1))
    ch2 = I.channel_chart(n, I.fourier_deformation(n, 2, 0.03, 42, True, kmax=1, lmax=1))
    L = oracle.Lattice(n, (P, P, P), tau=0.7, fext=(0, 0, 1e-4))
    L.set_metric(ch1.g6, ch1.dg18)
    L.init(1 + 0.05 * rng.standard_normal(N), 0.05 * rng.standard_normal((3, N)))
    L.step(5)  # a non-equilibrium state
    c, _ = oracle.lattice()
    sg1 = L.sqrtg.copy()
    a0 = (L.f * sg1).sum(0)
    a1 = np.einsum("ln,li->in", L.f * sg1, c)
    Pi = np.einsum("ln,li,lj->ijn", L.f * sg1, c, c)
    A = (L.Fprev * sg1).sum(0)
    B = np.einsum("ln,li->in", L.Fprev * sg1, c)
    # identity chart change = projection onto the 2nd-order Hermite space
    L.transform(ch1.g6, ch1.dg18, ch1.J9, ch1.J9)
    proj = L.f.copy()
    L.transform(ch1.g6, ch1.dg18, ch1.J9, ch1.J9)
    assert np.abs(L.f - proj).max() < 1e-15
    assert np.abs((L.f * sg1).sum(0) - a0).max() < 1e-14
    assert np.abs(np.einsum("ln,li,lj->ijn", L.f * sg1, c, c) - Pi).max() < 1e-14
    # a real chart change transforms a_(1), Pi and the history as tensors
    L.transform(ch2.g6, ch2.dg18, ch1.J9, ch2.J9)
    J1 = np.moveaxis(ch1.J9.reshape(3, 3, N), 2, 0)
    J2 = np.moveaxis(ch2.J9.reshape(3, 3, N), 2, 0)
    D = np.moveaxis(np.linalg.solve(J2, J1), 0, 2)
    sg2 = L.sqrtg
    assert np.abs((L.f * sg2).sum(0) - a0).max() < 1e-14
    assert np.abs(np.einsum("ln,li->in", L.f * sg2, c) - np.einsum("ijn,jn->in", D, a1)).max() < 1e-14
    assert np.abs(np.einsum("ln,li,lj->ijn", L.f * sg2, c, c)
                  - np.einsum("ikn,jln,kln->ijn", D, D, Pi)).max() < 1e-14
    assert np.abs((L.Fprev * sg2).sum(0) - A).max() < 1e-15
    assert np.abs(np.einsum("ln,li->in", L.Fprev * sg2, c) - np.einsum("ijn,jn->in", D, B)).max() < 1e-15


def test_transform_literal_mode_agrees_for_rotations():
    """Under an orthogonal D phi, delta is invariant, so transforming a_(2)
    itself or Pi gives the same result."""
    n = (4, 4, 4)
    N = int(np.prod(n))
    rng = np.random.default_rng(10)
    Q_, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Jold = np.zeros((9, N))
    Jold[[0, 4, 8]] = 1.0
    Jnew = np.repeat(Q_.T.reshape(9, 1), N, axis=1)  # D phi = Q
    flat = I.flat_chart(n)
    res = []
    for literal in (False, True):
        L = oracle.Lattice(n, (P, P, P), tau=0.7, literal_a2=literal)
        L.init(1 + 0.05 * rng.standard_normal(N) * 0, 0.05 * np.ones((3, N)))
        L.step(2)
        L.transform(flat.g6, flat.dg18, Jold, Jnew)
        res.append(L.f.copy())
    assert np.abs(res[0] - res[1]).max() < 1e-15


def test_curved_rest_spurious_velocity_small_and_shrinking():
    """A fluid at rest under a static deformed-channel metric (5 % amplitude)
    develops only a small steady spurious velocity from the O(dx^2) mismatch
    between the streamed pressure divergence and the forcing moment B; it
    shrinks under refinement at fixed amplitude (first order in lattice units,
    since the mismatch scales with the lattice pressure rho theta)."""
    peaks = []
    for s in (1, 2):
        n = (8 * s + 1, 1, 16 * s)
        lay = (0, 1, 2)  # walls across axis 0, flow along axis 2
        dfm = I.fourier_deformation(n, 1, 0.05, 0, True, modes=([1], [0], [-np.pi / 2]),
                                    coeffs=[1.0], layout=lay)
        ch = I.channel_chart(n, dfm, lay)
        L = oracle.Lattice(n, (W, P, P), (W, P, P), tau=0.8)
        L.set_metric(ch.g6, ch.dg18)
        L.init()
        L.step(300 * s * s)
        _, u = L.moments(ch.J9)
        peaks.append(np.abs(u).max())
    assert peaks[0] < 1e-3
    assert peaks[1] < peaks[0] / 1.6, peaks


@pytest.mark.parametrize("kind", ["stretch", "shear"])
def test_transform_literal_mode_under_stretch_and_shear(kind):
    """Literal-a2 reading of the transformation (Sec. IV.B): a_(2) = Pi -
    c_s^2 rho delta itself is mapped as a rank-2 tensor and f~ recomposed from
    (rho, D a_(1), D a_(2) D^T), so the new second moment is
    D (Pi - c_s^2 rho delta) D^T + c_s^2 rho delta; the forcing history follows
    the same rule with b2 = C - c_s^2 A delta.  Under a stretch or a shear
    D D^T != I, so this differs from the Pi-tensor reading (D Pi D^T), which
    the rotation pin cannot tell apart.  The new chart is h~ = M^-1 h, so
    D phi = J~^-1 J = J^-1 M J at every node."""
    n = (5, 4, 6)
    N = int(np.prod(n))
    M = np.diag([1.12, 0.91, 1.05]) if kind == "stretch" else np.array([[1.0, 0.25, 0.0], [0.0, 1.0, 0.0],
                                                                       [0.1, 0.0, 1.0]])
    Mi = np.linalg.inv(M)
    ch1 = I.channel_chart(n, I.fourier_deformation(n, 2, 0.03, 51, True, kmax=1, lmax=1))
    J1 = ch1.J9.reshape(3, 3, N)
    J2 = np.einsum("ab,bin->ain", Mi, J1)
    H2 = np.einsum("ab,bjkn->ajkn", Mi, ch1.hess.reshape(3, 3, 3, N))
    ch2 = I.Chart(n, J2.reshape(9, N), H2.reshape(27, N))
    c, _ = oracle.lattice()
    out = {}
    for literal in (False, True):
        L = oracle.Lattice(n, (P, P, P), tau=0.7, fext=(0, 2e-4, 1e-4), literal_a2=literal)
        L.set_metric(ch1.g6, ch1.dg18)
        L.init(1 + 0.02 * np.cos(np.arange(N)),
               0.04 * np.sin(np.arange(3 * N).reshape(3, N)))
        L.step(4)  # a non-equilibrium state with a non-zero history
        sg1 = L.sqrtg.copy()
        a0 = (L.f * sg1).sum(0)
        a1 = np.einsum("ln,li->in", L.f * sg1, c)
        Pi = np.einsum("ln,li,lj->ijn", L.f * sg1, c, c)
        A = (L.Fprev * sg1).sum(0)
        B = np.einsum("ln,li->in", L.Fprev * sg1, c)
        C = np.einsum("ln,li,lj->ijn", L.Fprev * sg1, c, c)
        L.transform(ch2.g6, ch2.dg18, ch1.J9, ch2.J9)
        sg2 = L.sqrtg
        D = np.moveaxis(np.linalg.solve(np.moveaxis(J2, 2, 0), np.moveaxis(J1, 2, 0)), 0, 2)
        dlt = np.eye(3)[:, :, None]
        Pi2 = np.einsum("ln,li,lj->ijn", L.f * sg2, c, c)
        C2 = np.einsum("ln,li,lj->ijn", L.Fprev * sg2, c, c)
        assert np.abs((L.f * sg2).sum(0) - a0).max() < 1e-14
        assert np.abs(np.einsum("ln,li->in", L.f * sg2, c) - np.einsum("ijn,jn->in", D, a1)).max() < 1e-14
        assert np.abs((L.Fprev * sg2).sum(0) - A).max() < 1e-15
        assert np.abs(np.einsum("ln,li->in", L.Fprev * sg2, c) - np.einsum("ijn,jn->in", D, B)).max() < 1e-15
        if literal:
            ref = np.einsum("ikn,jln,kln->ijn", D, D, Pi - CS2_ * a0 * dlt) + CS2_ * a0 * dlt
            refC = np.einsum("ikn,jln,kln->ijn", D, D, C - CS2_ * A * dlt) + CS2_ * A * dlt
        else:
            ref = np.einsum("ikn,jln,kln->ijn", D, D, Pi)
            refC = np.einsum("ikn,jln,kln->ijn", D, D, C)
        assert np.abs(Pi2 - ref).max() < 1e-14
        assert np.abs(C2 - refC).max() < 1e-15 + 1e-12 * np.abs(refC).max()
        out[literal] = Pi2
    # the two readings differ here by c_s^2 rho (delta - D D^T)
    assert np.abs(out[True] - out[False]).max() > 1e-3
