"""Reduced-precision storage against the FP64 oracle on a 64^3 run of the
precision-form generator (8 Fourier modes, seed 3000, dynamic metric
re-transformed every 10 steps under a(t) = sin^2(pi t / 2000), tau 0.6,
Re 100, inflow/outflow), 2000 steps: relative L2 error of density, Cartesian
velocity and the force on the deformed wall for FP32, FP16 and BF16
weight-shifted storage (FP32 arithmetic, FP64 reductions).

The amplitude is 4 % of the channel height.  At 8 % this field (wall slopes
near 2 where the modes add up) drives the second-order D3Q19 method unstable
next to the deformed wall after about 700 steps, in the FP64 oracle and on
the GPU alike, at every tau and Re tried (0.6-0.8, 50-100); at 4 % the run
stays subsonic for all 2000 steps.  The measured errors are printed; the
bounds asserted here are the stated accuracy of each storage format."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N3 = (64, 64, 64)
STEPS = 2000
EVERY = 10
# stated bounds (relative L2): density, velocity, wall force
BOUND = {"fp32": (1e-5, 1e-4, 1e-4), "fp16": (2e-3, 5e-2, 5e-2), "bf16": (2e-2, 2e-1, 2e-1)}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def run(make, w, steps):
    """Advance one lattice through the schedule: every EVERY steps the chart
    and face velocities of the generator at that time, the metric updated and
    the state transformed."""
    lat, upd, face = make()
    ch_old = w["chart"]
    for t in range(EVERY, steps + 1, EVERY):
        lat.step(EVERY)
        if t == steps:
            break
        ch, faces = I.dynamic_channel_at(w, float(t))
        upd(lat, ch, ch_old)
        for (axis, side), u in faces.items():
            face(lat, axis, side, u)
        ch_old = ch
    return lat, ch_old


@pytest.fixture(scope="module")
def workload():
    return I.dynamic_channel(n=N3, seed=3000, n_modes=8, amp=0.04, tau=0.6, re=100.0, period=2000.0)


@pytest.fixture(scope="module")
def reference(workload):
    w = workload

    def make():
        o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(w["chart"].g6, w["chart"].dg18)
        for (axis, side), u in w["faces"].items():
            o.set_face_velocity(axis, side, u)
        o.init()
        return (o, lambda lat, ch, old: lat.transform(ch.g6, ch.dg18, old.J9, ch.J9),
                lambda lat, a, s, u: lat.set_face_velocity(a, s, u))

    o, ch = run(make, w, STEPS)
    wa = w["layout"][0]
    return o.moments(ch.J9), o.wall_force(wa, 1, ch.J9)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_storage_error_against_oracle(workload, reference, storage):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    w = workload

    def make():
        g = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=storage)
        g.set_chart(w["chart"])
        for (axis, side), u in w["faces"].items():
            g.set_boundary_velocity(axis, side, u)
        g.init_equilibrium()
        return (g, lambda lat, ch, old: lat.update_metric(ch.g6, ch.dg18, ch.J9),
                lambda lat, a, s, u: lat.set_boundary_velocity(a, s, u))

    g, ch = run(make, w, STEPS)
    assert g.check()
    (ro, uo), fo = reference
    rg, ug = g.moments(cartesian=True)
    fg = g.wall_force(w["layout"][0], 1)
    er, eu, ef = rel(rg, ro), rel(ug, uo), rel(fg, fo)
    print(f"\n{storage}: rel L2 rho {er:.3e}  u {eu:.3e}  wall force {ef:.3e}")
    br, bu, bf = BOUND[storage]
    assert er < br and eu < bu and ef < bf, (storage, er, eu, ef)
