"""The chart change with its derivatives and Jacobian in FP32
(cslbm_update_metric_mixed): for FP32-arithmetic storage the library rounds
dg and J to FP32 before any use, so the state it leaves must be, bit for bit,
the one the FP64-input chart change leaves; FP64 storage and host arrays are
refused."""
import numpy as np
import pytest

from paper_1803_07822_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def lattice(w, storage):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    g = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=storage)
    g.set_chart(w["chart"])
    for (axis, side), u in w["faces"].items():
        g.set_boundary_velocity(axis, side, u)
    g.init_equilibrium()
    return g


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_mixed_chart_change_is_bitwise_the_fp64_one(storage):
    import torch
    w = I.dynamic_channel(n=(9, 45, 17), seed=2000, n_modes=6, amp=0.06, tau=0.6, re=20.0, period=400.0, kmax=2,
                          lmax=1)
    a, b = lattice(w, storage), lattice(w, storage)
    for t in (10.0, 20.0, 30.0):
        a.step(10)
        b.step(10)
        ch, _ = I.dynamic_channel_at(w, t)
        g6 = torch.as_tensor(ch.g6, device="cuda")
        a.update_metric(g6, torch.as_tensor(ch.dg18, device="cuda"), torch.as_tensor(ch.J9, device="cuda"))
        b.update_metric_mixed(g6, torch.as_tensor(ch.dg18, device="cuda").float(),
                              torch.as_tensor(ch.J9, device="cuda").float())
    a.step(5)
    b.step(5)
    assert a.check() and b.check()
    ra, ua = a.moments(cartesian=True)
    rb, ub = b.moments(cartesian=True)
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    assert np.abs(ua).max() > 1e-3
    # the whole state (populations and forcing history), byte for byte; the
    # masses agree to the rounding of their FP64 block sums, added in any order
    assert bool((a.save_state() == b.save_state()).all())
    assert abs(a.total_mass() - b.total_mass()) < 1e-12 * a.total_mass()


def test_mixed_chart_change_refuses_fp64_storage_and_host_arrays():
    import torch
    from paper_1803_07822_gb300._abi import CslbmError, call
    w = I.dynamic_channel(n=(9, 45, 17), seed=2000, n_modes=6, amp=0.06, tau=0.6, re=20.0, period=400.0, kmax=2,
                          lmax=1)
    ch = w["chart"]
    g64 = lattice(w, "fp64")
    with pytest.raises(CslbmError, match="EINVAL"):
        g64.update_metric_mixed(torch.as_tensor(ch.g6, device="cuda"), torch.as_tensor(ch.dg18, device="cuda"),
                                torch.as_tensor(ch.J9, device="cuda"))
    g32 = lattice(w, "fp32")
    g6 = np.ascontiguousarray(ch.g6)
    d = np.ascontiguousarray(ch.dg18, dtype=np.float32)
    J = np.ascontiguousarray(ch.J9, dtype=np.float32)
    with pytest.raises(CslbmError, match="EINVAL"):
        call("cslbm_update_metric_mixed", g32.ctx, g6.ctypes.data, d.ctypes.data, J.ctypes.data)
    assert g32.check()
