"""The benchmark's workloads at their full sizes, in the launch configuration
bench.py times, against the oracle: over the whole field, one cycle of the
128 x 128 x 256 dynamic channel (chart change with transformation, face
velocities, 10 steps through the default step pass, mass and wall force) and
5 steps of the 4096 x 1024 D2Q9 channel; on sampled windows, one cycle of the
256^3 channel in FP32, FP16 and BF16 storage."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_dynamic_channel_one_bench_cycle():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    b = _bench()
    spec = b.workload_spec("dynamic")
    w = I.dynamic_channel(n=spec["n"], seed=spec["seed"], n_modes=spec["n_modes"], amp=spec["amp"], tau=spec["tau"],
                          re=spec["re"])
    (ch0, f0), (ch1, f1) = b.snapshots(w, [500.0, 510.0])
    g = CurvedLattice(spec["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp32")
    o = oracle.Lattice(spec["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    g.set_chart(ch0)
    o.set_metric(ch0.g6, ch0.dg18)
    for (a, s), u in f0.items():
        g.set_boundary_velocity(a, s, u)
        o.set_face_velocity(a, s, u)
    g.init_equilibrium()
    o.init()
    g.step(10)
    o.step(10)
    g.update_metric(ch1.g6, ch1.dg18, ch1.J9)
    o.transform(ch1.g6, ch1.dg18, ch0.J9, ch1.J9)
    for (a, s), u in f1.items():
        g.set_boundary_velocity(a, s, u)
        o.set_face_velocity(a, s, u)
    g.step(10)
    o.step(10)
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(ch1.J9)
    print(f"\n128x128x256 dynamic channel, one cycle: rel L2 rho {rel(rg, ro):.2e}, u {rel(ug, uo):.2e}")
    assert rel(rg, ro) < 1e-5 and rel(ug, uo) < 1e-5
    assert abs(g.total_mass() - o.mass()) < 1e-6 * o.mass()
    Fg, Fo = g.wall_force(2, 1), o.wall_force(2, 1, ch1.J9)
    assert np.abs(Fg - Fo).max() < 1e-5 * np.abs(Fo).max()


def test_d2q9_bench_channel_five_steps():
    from paper_1803_07822_gb300.lattice import CurvedLattice2D
    n = (4096, 1024)
    H = n[1] - 1
    x = I.grid2d(n)[0]
    k = 2 * np.pi / n[0]
    a = 0.06 * H
    ch = I.channel_chart2d(n, a * np.cos(k * x), -a * k * np.sin(k * x), -a * k * k * np.cos(k * x))
    tau = 0.8
    F = 8.0 * (tau - 0.5) / 3.0 * 0.05 / H ** 2
    g = CurvedLattice2D(n, (0, 1), (0, 1), tau=tau, fext=(F, 0.0), storage="fp32")
    g.set_chart(ch)
    o = oracle.Lattice2D(n, (0, 1), (0, 1), tau=tau, fext=(F, 0.0))
    o.set_metric(ch.g3, ch.dg6)
    rng = np.random.default_rng(3)
    rho0 = 1 + 0.001 * rng.standard_normal(x.size)
    u0 = 0.01 * rng.standard_normal((2, x.size))
    g.init_equilibrium(rho0, u0)
    o.init(rho0, u0)
    g.step(5)
    o.step(5)
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(ch.J4)
    assert rel(rg, ro) < 1e-5 and rel(ug, uo) < 1e-5, (rel(rg, ro), rel(ug, uo))


def test_target_256_cube_sampled_windows():
    """The 256^3 deformed channel (8 modes, 8 % amplitude, parabolic inflow,
    outflow, moving top wall), one cycle of the bench schedule (10 steps,
    chart change with transformation, 10 steps) through the default pass, in
    FP32 and in FP16/BF16 weight-shifted storage, from a developed-flow state.
    The oracle cannot run the whole lattice here, so it runs windows around
    five sampled cores (interior, both walls, the inlet at the bottom wall,
    the outlet at the top wall); each window reproduces the whole run exactly
    on its core (tests/test_windows.py checks that on a small lattice)."""
    from paper_1803_07822_gb300.lattice import CurvedLattice
    from windows import Window, oracle_cycle
    b = _bench()
    spec = b.workload_spec("target256")
    n = spec["n"]
    w = I.dynamic_channel(n=n, seed=spec["seed"], n_modes=spec["n_modes"], amp=spec["amp"], tau=spec["tau"],
                          re=spec["re"])
    charts = b.snapshots(w, [500.0, 510.0])
    rho0, u0 = I.developed_flow(n, w["umax"], 17)
    steps = (10, 10)
    R = 3 * sum(steps) + 2
    core = 6

    def span(where, m):
        if where == "lo":
            return 0, core + R
        if where == "hi":
            return m - core - R, core + R
        return m // 2 - core // 2 - R, core + 2 * R

    # axes: 0 span (periodic), 1 flow (inflow low, outflow high), 2 wall-normal
    places = [("mid", "mid", "mid"), ("mid", "mid", "lo"), ("mid", "mid", "hi"), ("mid", "lo", "lo"),
              ("mid", "hi", "hi")]
    wins, ref = [], []
    for pl in places:
        lo, size = zip(*(span(pl[a], n[a]) for a in range(3)))
        win = Window(n, w["bc_lo"], w["bc_hi"], lo, size, R)
        rw, uw = oracle_cycle(n, w["bc_lo"], w["bc_hi"], w["tau"], charts, steps, win, rho0, u0)
        wins.append(win)
        ref.append((rw[win.core], uw[:, win.core]))
    ro = np.concatenate([r for r, _ in ref])
    uo = np.concatenate([u for _, u in ref], axis=1)
    assert np.abs(uo).max() > 0.01  # the flow is there
    (ch0, f0), (ch1, f1) = charts
    for storage, tol in (("fp32", 1e-5), ("fp16", 3e-2), ("bf16", 1e-1)):
        g = CurvedLattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=storage)
        g.set_chart(ch0)
        for (a, s), u in f0.items():
            g.set_boundary_velocity(a, s, u)
        g.init_equilibrium(rho0, u0)
        g.step(steps[0])
        g.update_metric(ch1.g6, ch1.dg18, ch1.J9)
        for (a, s), u in f1.items():
            g.set_boundary_velocity(a, s, u)
        g.step(steps[1])
        rg, ug = g.moments(cartesian=True)
        sel = np.concatenate([win.core_global for win in wins])
        er, eu = rel(rg[sel], ro), rel(ug[:, sel], uo)
        print(f"\n256^3 {storage}, {sel.size} sampled nodes: rel L2 rho {er:.2e}, u {eu:.2e}")
        assert er < tol and eu < tol, (storage, er, eu)
        del g
