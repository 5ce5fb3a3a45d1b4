"""Lattice derivatives on the GPU (App. D: isotropic gradient of order 2 and
4, the geometry from the metric alone) against the oracle's stencils, and
properties that hold at any size on the 128 x 256 x 128 bench channel."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I
from paper_1803_07822_gb300._abi import CslbmError, EINVAL

pytestmark = pytest.mark.gpu

P, W, IN, OUT = 0, 1, 2, 3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def lattice(n, lo, hi, storage="fp64"):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    return CurvedLattice(n, lo, hi, tau=0.8, storage=storage, step_kernel="flat")


CASES = [
    ("walls everywhere, ragged", (13, 10, 9), (W, W, W), (W, W, W)),
    ("periodic x, walls y, inflow/outflow z", (16, 9, 7), (P, W, IN), (P, W, OUT)),
    ("all periodic", (12, 10, 8), (P, P, P), (P, P, P)),
    ("five nodes across the walls", (6, 5, 5), (P, W, W), (P, W, W)),
]


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("name,n,lo,hi", CASES, ids=[c[0] for c in CASES])
def test_gradient_matches_oracle(name, n, lo, hi, order):
    N = int(np.prod(n))
    rng = np.random.default_rng(7)
    x = np.stack(np.meshgrid(*[np.arange(k) for k in n[::-1]], indexing="ij")[::-1]).reshape(3, -1)
    f = np.stack([np.sin(0.4 * x[0] + 0.2 * x[1]) * np.cos(0.3 * x[2]), rng.normal(size=N),
                  1.0 + 0.01 * x[0] * x[1] - 0.02 * x[2] ** 2])
    lat = lattice(n, lo, hi)
    g = lat.lattice_gradient(f, order).cpu().numpy()
    ref = oracle.lattice_gradient(n, f, order, bc_lo=lo, bc_hi=hi)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(g - ref).max()


def test_metric_from_lattice_drives_the_same_flow_as_the_oracle():
    """Geometry from g alone (fourth-order dg on the lattice), 200 FP32 steps,
    against the oracle fed the oracle's own fourth-order lattice dg (two
    resolved modes: the lattice dg is 9e-5 from the analytic one and moves
    u by 3e-4, far above the parity bar)."""
    w = I.periodic_channel((16, 32, 16), 0.8, 0.05, 2, 0.06, 11, kmax=1, lmax=1)
    ch = w["chart"]
    from paper_1803_07822_gb300.lattice import CurvedLattice
    lat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp32")
    lat.set_metric_lattice(ch.g6, 4)
    lat.set_jacobian(ch.J9)
    lat.init_equilibrium()
    lat.step(200)
    dg = oracle.lattice_gradient(w["n"], ch.g6, 4, bc_lo=w["bc_lo"], bc_hi=w["bc_hi"]).reshape(18, -1)
    o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(ch.g6, dg)
    o.init()
    o.step(200)
    rg, ug = lat.moments(cartesian=True)
    ro, uo = o.moments(ch.J9)
    assert rel(rg, ro) < 1e-5 and rel(ug, uo) < 1e-5, (rel(rg, ro), rel(ug, uo))
    # and the lattice dg is not the analytic one: the flows differ measurably
    o2 = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o2.set_metric(ch.g6, ch.dg18)
    o2.init()
    o2.step(200)
    assert rel(uo, o2.moments(ch.J9)[1]) > 1e-6


def test_update_metric_lattice_equals_update_with_supplied_derivative():
    from paper_1803_07822_gb300.lattice import CurvedLattice
    n = (16, 24, 12)
    w = I.periodic_channel(n, 0.7, 0.05, 3, 0.05, 12)
    ch0 = w["chart"]
    ch1 = I.channel_chart(n, w["dfm"].scaled(1.3), w["layout"])
    dg1 = oracle.lattice_gradient(n, ch1.g6, 2, bc_lo=w["bc_lo"], bc_hi=w["bc_hi"]).reshape(18, -1)
    runs = []
    for mode in ("lattice", "supplied"):
        lat = CurvedLattice(n, w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp64")
        lat.set_chart(ch0)
        lat.init_equilibrium()
        lat.step(20)
        if mode == "lattice":
            lat.update_metric_lattice(ch1.g6, ch1.J9, 2)
        else:
            lat.update_metric(ch1.g6, dg1, ch1.J9)
        lat.step(20)
        runs.append(lat.moments())
    assert rel(runs[0][0], runs[1][0]) < 1e-12 and rel(runs[0][1], runs[1][1]) < 1e-10


def test_bench_channel_properties():
    """128 x 256 x 128 (span, flow, wall; walls, inflow/outflow): quartic
    fields are differentiated exactly at order 4, and on the dynamic chart's
    metric the order-4 error against the analytic dg is below the order-2 one."""
    n = (128, 256, 128)
    w = I.dynamic_channel(n=n, t=500.0)
    lat = lattice(n, w["bc_lo"], w["bc_hi"])
    x = np.stack(np.meshgrid(*[np.arange(k, dtype=float) for k in n[::-1]], indexing="ij")[::-1]).reshape(3, -1)
    s = 1.0 / 128
    q = (s * x[0]) ** 4 - 2 * (s * x[1]) ** 3 * (s * x[2]) + (s * x[2]) ** 2 + 0.5 * (s * x[0]) * (s * x[1])
    dq = np.stack([s * (4 * (s * x[0]) ** 3 + 0.5 * s * x[1]), s * (-6 * (s * x[1]) ** 2 * (s * x[2]) + 0.5 * s * x[0]),
                   s * (-2 * (s * x[1]) ** 3 + 2 * s * x[2])])
    lat_w = lattice(n, (W, W, W), (W, W, W))
    g = lat_w.lattice_gradient(q, 4).cpu().numpy()[:, 0]
    assert rel(g, dq) < 1e-10
    ch = w["chart"]
    e = [rel(lat.lattice_gradient(ch.g6, k).cpu().numpy().reshape(18, -1), ch.dg18) for k in (2, 4)]
    print(f"\n128x256x128 dynamic chart: dg rel err order 2 {e[0]:.2e}, order 4 {e[1]:.2e}")
    assert e[1] < 0.5 * e[0]


def test_errors():
    lat = lattice((4, 6, 4), (P, W, W), (P, W, W))
    f = np.zeros((1, lat.N))
    with pytest.raises(CslbmError) as ex:
        lat.lattice_gradient(f, 3)
    assert ex.value.status == EINVAL
    with pytest.raises(CslbmError) as ex:
        lat.lattice_gradient(f, 4)  # 4 nodes across the walls: order 4 needs 5
    assert ex.value.status == EINVAL
    assert np.abs(lat.lattice_gradient(f, 2).cpu().numpy()).max() == 0.0
    # host memory through the raw ABI
    import ctypes

    from paper_1803_07822_gb300._abi import call
    import torch
    out = torch.empty((3, lat.N), dtype=torch.float64, device="cuda")
    nb = ctypes.c_size_t(0)
    call("cslbm_lattice_gradient_scratch_bytes", lat.ctx, 1, 2, ctypes.byref(nb))
    scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    with pytest.raises(CslbmError) as ex:
        call("cslbm_lattice_gradient", lat.ctx, f.ctypes.data_as(ctypes.c_void_p), 1, 2, out.data_ptr(),
             scratch.data_ptr(), nb.value)
    assert ex.value.status == EINVAL
    with pytest.raises(CslbmError) as ex:  # a short scratch
        call("cslbm_lattice_gradient", lat.ctx, torch.zeros(lat.N, dtype=torch.float64, device="cuda").data_ptr(), 1,
             2, out.data_ptr(), scratch.data_ptr(), nb.value - 8)
    assert ex.value.status == 3  # ENOMEM
