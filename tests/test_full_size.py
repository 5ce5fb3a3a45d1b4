"""The benchmark's workloads at their full sizes, in the launch configuration
bench.py times, against the oracle: over the whole field (and over each
non-periodic face plane and the interior on its own), one cycle of the
128 x 128 x 256 dynamic channel from a developed flow (10 steps, chart change
with transformation, face velocities, 10 steps through the default step
pass, mass and wall force) and
5 steps of the 4096 x 1024 D2Q9 channel.  The 256^3 channel and the full
64-channel batch are in test_full_size_sampled.py."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I
from planes import assert_regions

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
    # from a developed flow, so that the velocity on every plane (the outlet
    # included) is well above FP32 rounding from the first step
    rho0, u0 = I.developed_flow(spec["n"], w["umax"], 17)
    g.init_equilibrium(rho0, u0)
    o.init(rho0, u0)
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
    errs = assert_regions(rg, ug, ro, uo, spec["n"], w["bc_lo"], w["bc_hi"], 1e-5, "128x128x256")
    print("  " + ", ".join(f"{k}: rho {v[0]:.1e} u {v[1]:.1e}" for k, v in errs.items()))
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

