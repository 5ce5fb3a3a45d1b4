"""The fused step pass's bounded waits, made to run out on purpose.

The fused pass synchronises its CTAs through per-iteration publication
counts; every wait in it gives up after a limit, sets the context's error
flag and lets the kernel return, and cslbm_check reports CSLBM_ETIMEOUT and
resets the counts.  cslbm_test_withhold_publication makes the next fused
launch leave one momentum iteration of CTA 0 uncounted under a 1 ms limit,
so that every step tile waiting on it times out.  The tests check the
status, that the counts were reset (the next steps run clean), and that the
lattice then matches an untouched twin bit for bit and the oracle within the
FP32 bar.  Two lattices: one iteration per CTA (a tile's dependency times
out on its last tile) and two (the later tile is never issued and the
compute warps' stage wait runs out too)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import _abi
from paper_1803_07822_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W, P = oracle.WALL, oracle.PERIODIC


def channel(n):
    dfm = I.fourier_deformation(n, 2, 0.04, seed=9, flow_periodic=True, kmax=1, lmax=1)
    ch = I.channel_chart(n, dfm)
    return dict(n=n, bc_lo=(P, P, W), bc_hi=(P, P, W), tau=0.7, fext=(0.0, 2e-4, 0.0), chart=ch)


def lattice(w):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    g = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp32")
    g.set_chart(w["chart"])
    g.init_equilibrium()
    return g


@pytest.mark.parametrize("n", [(32, 16, 12), (32, 64, 40)], ids=["one iteration per CTA", "two iterations"])
def test_withheld_publication_times_out_and_recovers(n):
    lib = _abi.load()
    w = channel(n)
    g, twin = lattice(w), lattice(w)
    g.step(5)
    twin.step(5)
    snap = g.save_state()
    assert lib.cslbm_test_withhold_publication(g.ctx, 0, ctypes.c_longlong(1_000_000)) == _abi.OK
    g.step(1)
    st = lib.cslbm_check(g.ctx)
    assert st == _abi.ETIMEOUT, (st, lib.cslbm_last_error())
    assert b"bounded wait" in lib.cslbm_last_error()
    # the flag and the counts were reset; the hook applied to one launch only
    g.load_state(snap)
    assert lib.cslbm_check(g.ctx) == _abi.OK
    g.step(20)
    twin.step(20)
    assert lib.cslbm_check(g.ctx) == _abi.OK
    rg, ug = g.moments(cartesian=True)
    rt, ut = twin.moments(cartesian=True)
    assert np.array_equal(rg, rt) and np.array_equal(ug, ut)
    o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(w["chart"].g6, w["chart"].dg18)
    o.init()
    o.step(25)
    ro, uo = o.moments(w["chart"].J9)
    assert np.linalg.norm(rg - ro) / np.linalg.norm(ro) < 1e-5
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-5


def test_hook_refused_where_the_fused_pass_does_not_apply():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    lib = _abi.load()
    w = channel((32, 16, 12))
    flat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp64")
    assert lib.cslbm_test_withhold_publication(flat.ctx, 0, ctypes.c_longlong(1_000_000)) == _abi.EINVAL
    g = lattice(w)
    assert lib.cslbm_test_withhold_publication(g.ctx, -1, ctypes.c_longlong(1_000_000)) == _abi.EINVAL
    assert lib.cslbm_test_withhold_publication(g.ctx, 0, ctypes.c_longlong(0)) == _abi.EINVAL
    assert lib.cslbm_test_withhold_publication(g.ctx, 0, ctypes.c_longlong(10 ** 9)) == _abi.EINVAL
