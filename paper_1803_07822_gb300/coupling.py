"""Host-side coupled loop with a prescribed-motion shell (the flow chart of
Sec. III: update the geometry, transform f, step, pass T.n out, take the wall
velocity in), for a rigid piston: the top wall of a box pressed down by d(t)
(Sec. V.B piston test).  A caller of the library: the chart of every step is
the channel chart with a uniform displacement d(t) of the top wall, the
transformation is the node-wise one, the top wall moves with velocity d'(t).
"""
from __future__ import annotations

import numpy as np

from . import inputs as I

THETA = 1.0 / 3.0


def piston_chart(n, d, layout=I.LAYOUT):
    """Channel chart h^w = x_w (1 + d/H) with a uniform displacement d of the
    top wall (no variation along the wall: all Christoffel symbols vanish)."""
    N = int(np.prod(n))
    z = np.zeros(N)
    return I.channel_chart(n, I.Deformation(np.full(N, float(d)), z, z, z, z, z), layout)


def piston_law(t, T, amp, H):
    """d(t) = -amp H (1 - cos(pi t / T)) / 2 for t <= T, then held: a smooth
    press by amp H; returns (d, d')."""
    if t >= T:
        return -amp * H, 0.0
    a = np.pi / T
    return -amp * H * 0.5 * (1.0 - np.cos(a * t)), -amp * H * 0.5 * a * np.sin(a * t)


def run_piston(n=(16, 16, 32), steps=2000, T=1000, amp=0.002, tau=0.8, storage="fp32", sample=50,
               layout=I.LAYOUT):
    """Runs the loop; returns time series every `sample` steps: mass (sum
    sqrt(g) rho), volume (sum sqrt(g)), mean density, Cartesian momentum
    (sum sqrt(g) rho v), the force on the piston, and the impulse on the
    piston (sum of the force over the steps) next to sum p A with p = mean
    density x theta, A the piston's node count."""
    from .lattice import CurvedLattice
    w = layout[0]
    H = n[w] - 1
    lo = [0, 0, 0]
    lo[w] = 1
    lat = CurvedLattice(n, tuple(lo), tuple(lo), tau=tau, storage=storage)
    ch = piston_chart(n, 0.0, layout)
    lat.set_chart(ch)
    lat.init_equilibrium()
    nf = lat.face_nodes(w)
    A = float(nf)
    out = {k: [] for k in ("t", "mass", "volume", "rho_mean", "momentum", "force", "impulse", "impulse_pA")}
    impulse = np.zeros(3)
    impulse_pa = 0.0
    for t in range(steps):
        d, dd = piston_law(float(t), T, amp, H)
        if t > 0:
            ch = piston_chart(n, d, layout)
            lat.update_metric(ch.g6, ch.dg18, ch.J9)
        Jww = 1.0 + d / H
        u3 = np.zeros((3, nf))
        u3[w] = dd / Jww  # contravariant wall velocity of the piston
        lat.set_boundary_velocity(w, 1, u3)
        lat.step(1)
        F = lat.wall_force(w, 1)
        sg = np.prod([ch.J9[a * 3 + a] for a in range(3)], axis=0)
        vol = float(sg.sum())
        if t % sample == 0 or t == steps - 1:
            rho, v = lat.moments(cartesian=True)
            m = float((sg * rho).sum())
            out["t"].append(t + 1)
            out["mass"].append(m)
            out["volume"].append(vol)
            out["rho_mean"].append(m / vol)
            out["momentum"].append((sg * rho * v).sum(axis=1))
            out["force"].append(F)
        # the impulse and its pressure-area estimate, every step
        impulse += F
        impulse_pa += lat.total_mass() / vol * THETA * A
        if t % sample == 0 or t == steps - 1:
            out["impulse"].append(impulse.copy())
            out["impulse_pA"].append(impulse_pa)
    lat.close()
    return {k: np.array(v) for k, v in out.items()}
