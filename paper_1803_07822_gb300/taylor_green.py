"""The Taylor-Green vortex under a dynamic periodic metric (the paper's
dynamic-metric validation, Sec. V.A): a caller of the library that builds the
chart at every time (``inputs.tg_chart``), starts from the analytic field and
changes the chart every ``every`` steps, by the interpolating transformation
(``update_metric_interp`` with the transition map ``inputs.tg_psi``) or the
node-wise one (``update_metric``), and compares the Cartesian velocity at the
nodes' current positions with the analytic decay.

Acoustic scaling across resolutions: the Mach number is fixed (v0 in lattice
units), tau follows from Re = v0 L / nu, the run ends at nu k^2 t = 0.5 (a
number of steps proportional to L), and the chart's angular rate is eta =
eta_ref L_ref / L, so every resolution sees the same motion of the chart over
the run.  (The second-order curved-space method has an O(dx) spurious
velocity at rest under a curved metric; under diffusive scaling v0 shrinks as
fast, so only acoustic scaling shows convergence.)
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def run(L, mode="interp", storage="fp64", v0=0.04, re=20.0, eps=0.1, eta_ref=0.05, L_ref=32, every=1, nz=4,
        t_end=0.5, step_kernel="flat"):
    """(relative L2 error of the Cartesian velocity against the analytic
    decay, the final Cartesian velocity [3, N], the steps taken).  mode:
    "interp" (interpolating transformation), "node" (node-wise) or "static"
    (the chart of t = 0 throughout); eps = 0 is the flat chart."""
    from .lattice import CurvedLattice
    n = (L, L, nz)
    nu = v0 * L / re
    tau = 0.5 + 3.0 * nu
    k = 2 * np.pi / L
    steps = int(round(t_end / (nu * k * k)))
    eta = eta_ref * L_ref / L
    lat = CurvedLattice(n, (0, 0, 0), (0, 0, 0), tau=tau, storage=storage, step_kernel=step_kernel)
    ch = I.tg_chart(n, 0.0, eps, eta)
    lat.set_chart(ch)
    rho, v = I.tg_velocity(I.tg_position(n, 0.0, eps, eta), L, v0, nu, 0.0)
    u = np.stack([v[a] / ch.J9[a * 3 + a] for a in range(3)])  # contravariant: u^i = (J^-1)^i_a v^a
    lat.init_equilibrium(rho, u)
    t, t_chart = 0, 0.0
    while t < steps:
        m = min(every, steps - t)
        lat.step(m)
        t += m
        if t < steps and mode != "static" and eps != 0.0:
            ch_new = I.tg_chart(n, float(t), eps, eta)
            if mode == "interp":
                lat.update_metric_interp(ch_new.g6, ch_new.dg18, ch_new.J9, I.tg_psi(n, t_chart, float(t), eps, eta))
            else:
                lat.update_metric(ch_new.g6, ch_new.dg18, ch_new.J9)
            t_chart = float(t)
    _, vg = lat.moments(cartesian=True)
    _, va = I.tg_velocity(I.tg_position(n, t_chart, eps, eta), L, v0, nu, float(steps))
    err = float(np.linalg.norm(vg[:2] - va[:2]) / np.linalg.norm(va[:2]))
    lat.close()
    return err, vg, steps
