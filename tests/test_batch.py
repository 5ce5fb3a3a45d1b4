"""Batched form: independent channels of uneven sizes advanced by one
persistent launch per step (work-item queue, grid barrier, CUDA graph),
against the FP64 oracle channel by channel and against the same channels
stepped one by one; the tile-shape tuner."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def small_batch(nb=6):
    # uneven sides 12..24 (ragged for every block size), one wavelength per
    # axis at most so that these short channels resolve their deformation
    return I.batch_channels(nb=nb, seed0=4100, side=(12, 24), kmax=1, lmax=1)


def make_batch(ws):
    from paper_1803_07822_gb300.lattice import CurvedBatch
    b = CurvedBatch([dict(n=w["n"], bc_lo=w["bc_lo"], bc_hi=w["bc_hi"], tau=w["tau"], fext=w["fext"]) for w in ws])
    for i, w in enumerate(ws):
        b[i].set_chart(w["chart"])
        b[i].init_equilibrium()
    return b


def test_batch_channels_match_oracle():
    ws = small_batch()
    b = make_batch(ws)
    b.step(61)  # 30 graph replays and one eager step
    for i in (0, 2, 5):
        w = ws[i]
        o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
        o.set_metric(w["chart"].g6, w["chart"].dg18)
        o.init()
        o.step(61)
        rg, ug = b[i].moments(cartesian=True)
        ro, uo = o.moments(w["chart"].J9)
        assert rel(rg, ro) < 1e-5 and rel(ug, uo) < 1e-5, (i, rel(rg, ro), rel(ug, uo))
        assert abs(b[i].total_mass() - o.mass()) / o.mass() < 1e-6


def test_batch_equals_channels_stepped_alone_with_metric_update():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    ws = small_batch(5)
    b = make_batch(ws)
    solo = []
    for w in ws:
        g = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], step_kernel="flat")
        g.set_chart(w["chart"])
        g.init_equilibrium()
        solo.append(g)
    b.step(7)
    for g in solo:
        g.step(7)
    # a chart change on one channel between batch steps (the batch's tables follow)
    w = ws[3]
    ch = I.channel_chart(w["n"], w["dfm"].scaled(1.2), w["layout"])
    b[3].update_metric(ch.g6, ch.dg18, ch.J9)
    solo[3].update_metric(ch.g6, ch.dg18, ch.J9)
    b.step(12)
    for g in solo:
        g.step(12)
    for i in range(len(ws)):
        r1, u1 = b[i].moments()
        r2, u2 = solo[i].moments()
        assert rel(r1, r2) < 1e-6 and rel(u1, u2) < 1e-5, i
    assert b.launches() == 19  # one persistent launch per step
    assert b.check()


def test_tune_picks_a_tile_shape_and_keeps_the_state():
    ws = small_batch(4)
    b = make_batch(ws)
    b.step(3)
    before = [c.moments() for c in b]
    shape, table = b.tune(reps=3)
    assert shape in table and len(table) >= 9
    assert {s[0] for s in table} == {128, 256, 512} and all(v > 0 for v in table.values())
    assert all(s[1] % s[0] == 0 and s[2] >= 1 for s in table)
    assert table[shape] == min(table.values())
    after = [c.moments() for c in b]
    for (r1, u1), (r2, u2) in zip(before, after):
        assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
    # every shape steps the same state to the same result
    from paper_1803_07822_gb300.lattice import CurvedBatch  # noqa: F401
    b.step(2)
    assert all(c.check() for c in b) and b.check()


@pytest.mark.parametrize("shape_index", [0, -1])
def test_batch_result_does_not_depend_on_the_tile_shape(shape_index):
    """The work-item queue hands out runs of nodes in any order and size; the
    per-node arithmetic is the same, so two tile shapes give the same bits."""
    ws = small_batch(4)
    a, c = make_batch(ws), make_batch(ws)
    _, table = a.tune(reps=1)
    shapes = sorted(table)
    a.set_shape(shapes[shape_index])
    c.set_shape(shapes[len(shapes) // 2])
    a.step(9)
    c.step(9)
    for i in range(len(ws)):
        r1, u1 = a[i].moments()
        r2, u2 = c[i].moments()
        assert np.array_equal(r1, r2) and np.array_equal(u1, u2), i
