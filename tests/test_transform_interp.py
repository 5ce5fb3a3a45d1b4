"""Chart change with interpolation on the GPU (Sec. IV.B transition maps)
against the oracle, and the Taylor-Green vortex under a dynamic periodic
metric (the paper's dynamic-metric validation) with both transformations."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I
from paper_1803_07822_gb300._abi import CslbmError, EINVAL, ENOMEM, ESTATE

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def channel_psi(n, w, dfm_old, dfm_new):
    """Old lattice coordinates of the new nodes' points under the channel
    chart h^w = x_w (1 + d / H): x_w = x~_w (1 + d~/H) / (1 + d/H)."""
    wax = w["layout"][0]
    H = n[wax] - 1
    psi = np.stack(I.grid(n))
    psi[wax] = psi[wax] * (1.0 + dfm_new.d / H) / (1.0 + dfm_old.d / H)
    return psi


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_channel_chart_change_matches_oracle(storage):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    n = (12, 16, 10)
    w = I.periodic_channel(n, 0.7, 0.05, 2, 0.06, 31, kmax=1, lmax=1)
    d0, d1 = w["dfm"], w["dfm"].scaled(1.5)
    ch0, ch1 = w["chart"], I.channel_chart(n, d1, w["layout"])
    psi = channel_psi(n, w, d0, d1)
    g = CurvedLattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=storage, step_kernel="flat")
    g.set_chart(ch0)
    g.init_equilibrium()
    g.step(12)
    g.update_metric_interp(ch1.g6, ch1.dg18, ch1.J9, psi)
    g.step(12)
    o = oracle.Lattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(ch0.g6, ch0.dg18)
    o.init()
    o.step(12)
    o.transform_interp(ch1.g6, ch1.dg18, ch0.J9, ch1.J9, psi)
    o.step(12)
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(ch1.J9)
    assert rel(rg, ro) < TOL[storage] and rel(ug, uo) < TOL[storage], (rel(rg, ro), rel(ug, uo))


@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_taylor_green_chart_sequence_matches_oracle(storage):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    n, L, eta = (16, 12, 4), 16, 0.2
    ch = I.tg_chart(n, 0.0, eta=eta)
    rho, v = I.tg_velocity(I.tg_position(n, 0.0, eta=eta), L, 0.03, 0.1, 0.0)
    u = np.stack([v[a] / ch.J9[a * 3 + a] for a in range(3)])
    g = CurvedLattice(n, (0, 0, 0), (0, 0, 0), tau=0.8, storage=storage, step_kernel="flat")
    g.set_chart(ch)
    g.init_equilibrium(rho, u)
    o = oracle.Lattice(n, (0, 0, 0), (0, 0, 0), tau=0.8)
    o.set_metric(ch.g6, ch.dg18)
    o.init(rho, u)
    for t in range(1, 9):
        g.step(2)
        o.step(2)
        c_new = I.tg_chart(n, 2.0 * t, eta=eta)
        psi = I.tg_psi(n, 2.0 * (t - 1), 2.0 * t, eta=eta)
        g.update_metric_interp(c_new.g6, c_new.dg18, c_new.J9, psi)
        o.transform_interp(c_new.g6, c_new.dg18, ch.J9, c_new.J9, psi)
        ch = c_new
    g.step(3)
    o.step(3)
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(ch.J9)
    assert rel(rg, ro) < TOL[storage] and rel(ug, uo) < TOL[storage], (rel(rg, ro), rel(ug, uo))


def test_identity_map_equals_node_wise_update():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    n = (10, 14, 8)
    w = I.periodic_channel(n, 0.7, 0.05, 2, 0.05, 41, kmax=1, lmax=1)
    ch1 = I.channel_chart(n, w["dfm"].scaled(0.6), w["layout"])
    out = []
    for interp in (True, False):
        g = CurvedLattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp64", step_kernel="flat")
        g.set_chart(w["chart"])
        g.init_equilibrium()
        g.step(9)
        if interp:
            g.update_metric_interp(ch1.g6, ch1.dg18, ch1.J9, np.stack(I.grid(n)))
        else:
            g.update_metric(ch1.g6, ch1.dg18, ch1.J9)
        g.step(9)
        out.append(g.moments())
    assert rel(out[0][0], out[1][0]) < 1e-13 and rel(out[0][1], out[1][1]) < 1e-12


def test_errors():
    import ctypes

    import torch

    from paper_1803_07822_gb300._abi import call
    from paper_1803_07822_gb300.lattice import CurvedLattice
    n = (6, 6, 6)
    g = CurvedLattice(n, (0, 0, 0), (0, 0, 0), tau=0.8, storage="fp32")
    ch = I.flat_chart(n)
    dev = {k: torch.as_tensor(getattr(ch, k), device="cuda") for k in ("g6", "dg18", "J9")}
    psi = torch.as_tensor(np.stack(I.grid(n)), device="cuda")
    nb = ctypes.c_size_t(0)
    call("cslbm_transform_interp_scratch_bytes", g.ctx, ctypes.byref(nb))
    scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    args = (dev["g6"].data_ptr(), dev["dg18"].data_ptr(), dev["J9"].data_ptr(), psi.data_ptr())
    g.set_chart(ch)
    with pytest.raises(CslbmError) as ex:  # before init
        call("cslbm_update_metric_interp", g.ctx, *args, scratch.data_ptr(), nb.value)
    assert ex.value.status == ESTATE
    g.init_equilibrium()
    with pytest.raises(CslbmError) as ex:
        call("cslbm_update_metric_interp", g.ctx, *args, scratch.data_ptr(), nb.value - 4)
    assert ex.value.status == ENOMEM
    host_psi = np.stack(I.grid(n))
    with pytest.raises(CslbmError) as ex:
        call("cslbm_update_metric_interp", g.ctx, *args[:3], host_psi.ctypes.data_as(ctypes.c_void_p),
             scratch.data_ptr(), nb.value)
    assert ex.value.status == EINVAL
    call("cslbm_update_metric_interp", g.ctx, *args, scratch.data_ptr(), nb.value)
    g.step(2)
    assert g.check()


def test_taylor_green_dynamic_metric_convergence():
    """Velocity error against the analytic decay at nu k^2 t = 0.5 for L = 16,
    32, 64, 128 (acoustic scaling: Re 20, Ma 0.07; eps 0.1, the chart turning
    by the same phase at every L).  The flat chart sets the floor of the
    method at this Mach number; a static curved chart converges to it; under
    the moving chart the interpolating transformation converges (first order:
    a trilinear re-sampling every step), and the node-wise one, which leaves
    the nodes' motion uncorrected, stays several times larger."""
    from paper_1803_07822_gb300 import taylor_green as TG
    Ls = [16, 32, 64, 128]
    rows = {L: {"flat": TG.run(L, "static", eps=0.0)[0], **{m: TG.run(L, m)[0] for m in ("static", "interp", "node")}}
            for L in Ls}
    slope = lambda key: float(np.polyfit(np.log(Ls), np.log([rows[L][key] for L in Ls]), 1)[0])
    print("\nTaylor-Green, dynamic metric (relative L2 error of v at nu k^2 t = 0.5), L =", Ls)
    for key in ("flat", "static", "interp", "node"):
        print(f"  {key:7s}", " ".join(f"{rows[L][key]:.2e}" for L in Ls), f" slope {slope(key):.2f}")
    assert rows[128]["static"] < 1.2 * rows[128]["flat"]
    assert slope("interp") < -0.7
    assert rows[128]["node"] > 3 * rows[128]["interp"]
