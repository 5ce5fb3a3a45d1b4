"""The windowed oracle (tests/windows.py) against the oracle on the whole
lattice: on a dynamic channel (walls, parabolic inflow, outflow, a moving
top wall, a chart change between two runs of steps), windows in the
interior, on the walls, at the inlet and in the corners reproduce the whole
run exactly on their cores; a radius below the bound does not."""
import numpy as np
import pytest

from paper_1803_07822_gb300 import inputs as I
from windows import Window, oracle_cycle

N3 = (36, 44, 34)
K1, K2 = 1, 1


def _run(n, bc_lo, bc_hi, tau, charts, win=None):
    rho0, u0 = I.developed_flow(n, 0.04, 5)
    return oracle_cycle(n, bc_lo, bc_hi, tau, charts, (K1, K2), win, rho0, u0)


@pytest.fixture(scope="module")
def case():
    w = I.dynamic_channel(n=N3, seed=7, n_modes=4, amp=0.08, tau=0.6, re=60.0, t=500.0)
    charts = [I.dynamic_channel_at(w, t) for t in (500.0, 510.0)]
    full = _run(N3, w["bc_lo"], w["bc_hi"], w["tau"], charts)
    return w, charts, full


BOXES = [((8, 12, 9), (20, 20, 19)),    # interior
         ((4, 10, 0), (20, 20, 12)),    # bottom wall
         ((0, 8, 22), (36, 20, 12)),    # top (moving) wall, whole span
         ((6, 0, 8), (20, 12, 18)),     # inlet
         ((0, 32, 22), (36, 12, 12))]   # outlet / top wall corner, whole span


@pytest.mark.parametrize("lo,size", BOXES)
def test_window_core_equals_whole_run(case, lo, size):
    w, charts, (rf, uf) = case
    R = 3 * (K1 + K2) + 2
    win = Window(N3, w["bc_lo"], w["bc_hi"], lo, size, R)
    rw, uw = _run(N3, w["bc_lo"], w["bc_hi"], w["tau"], charts, win)
    assert win.core.size > 0
    assert np.abs(rw[win.core] - rf[win.core_global]).max() < 1e-15
    assert np.abs(uw[:, win.core] - uf[:, win.core_global]).max() < 1e-17


def test_too_small_radius_is_seen(case):
    w, charts, (rf, uf) = case
    lo, size = BOXES[1]
    win = Window(N3, w["bc_lo"], w["bc_hi"], lo, size, 2)
    rw, uw = _run(N3, w["bc_lo"], w["bc_hi"], w["tau"], charts, win)
    assert np.abs(uw[:, win.core] - uf[:, win.core_global]).max() > 1e-12
