"""The heaviest full-size parity tests (marked late: run after the others): the 256^3
deformed channel through one bench cycle in FP32, FP16 and BF16 storage
against the oracle on sampled windows (tests/windows.py), and the benchmark's
64-channel batch in its launch configuration against the oracle on three
whole channels.  Each holds tens of GB of host memory for its inputs."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.late]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_batch(ws):
    from paper_1803_07822_gb300.lattice import CurvedBatch
    b = CurvedBatch([dict(n=w["n"], bc_lo=w["bc_lo"], bc_hi=w["bc_hi"], tau=w["tau"], fext=w["fext"]) for w in ws])
    for i, w in enumerate(ws):
        b[i].set_chart(w["chart"])
        b[i].init_equilibrium()
    return b


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


def test_full_batch_of_64_sampled_channels():
    """The benchmark's batch at its full size and in its launch
    configuration: 64 channels with sides drawn from U{32..96}, 4-mode
    deformations of 2-10 %, tau in [0.55, 1.0], the tile shape picked by the
    autotuner, one persistent launch per step replayed from the CUDA graph;
    20 steps from a
    developed-flow state (so that u is well conditioned), then the smallest,
    the largest and one more channel against the oracle over the whole
    channel, with mass."""
    ws = I.batch_channels(nb=64, seed0=4000)
    b = make_batch(ws)
    init = []
    for i, w in enumerate(ws):
        rho0, u0 = I.developed_flow(w["n"], 0.05, 100 + i)
        b[i].init_equilibrium(rho0, u0)
        init.append((rho0, u0))
    b.tune(reps=2)
    b.step(20)
    sizes = [int(np.prod(w["n"])) for w in ws]
    for i in sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17}):
        w = ws[i]
        o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(w["chart"].g6, w["chart"].dg18)
        o.init(*init[i])
        o.step(20)
        rg, ug = b[i].moments(cartesian=True)
        ro, uo = o.moments(w["chart"].J9)
        assert np.abs(uo).max() > 0.02
        assert rel(rg, ro) < 1e-5 and rel(ug, uo) < 1e-5, (i, w["n"], rel(rg, ro), rel(ug, uo))
        assert abs(b[i].total_mass() - o.mass()) / o.mass() < 1e-6
