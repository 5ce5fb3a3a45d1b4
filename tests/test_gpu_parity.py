"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Same seeded inputs on both sides; element-by-element comparison of density
and velocity (relative L2 over all nodes, and over each non-periodic face
plane and the interior on its own), mass and wall force.  Bars:
FP64 storage 1e-11, FP32 storage 1e-5 (the method's FP32 target after 1000
steps), FP16/BF16 weight-shifted storage a stated bound.  Sizes are odd and
ragged on purpose (not multiples of the kernels' tiles).
"""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I
from planes import assert_regions

pytestmark = pytest.mark.gpu

W, P, IN, OUT = oracle.WALL, oracle.PERIODIC, oracle.INFLOW, oracle.OUTFLOW


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def make_pair(w, storage, literal=False, step_kernel="auto"):
    from paper_1803_07822_gb300.lattice import CurvedLattice
    kw = dict(tau=w["tau"], fext=w["fext"])
    g = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], storage=storage, literal_a2=literal, step_kernel=step_kernel,
                      **kw)
    o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], literal_a2=literal, **kw)
    ch = w["chart"]
    g.set_chart(ch)
    o.set_metric(ch.g6, ch.dg18)
    for (axis, side), u in w.get("faces", {}).items():
        g.set_boundary_velocity(axis, side, u)
        o.set_face_velocity(axis, side, u)
    return g, o


def compare(g, o, J9, tol, tag=""):
    """All-node relative L2 of rho and of the Cartesian velocity, and the same
    over each non-periodic face plane and the interior, each under tol."""
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(J9)
    er, eu = rel(rg, ro), rel(ug, uo)
    assert np.isfinite(ug).all()
    assert er < tol and eu < tol, f"{tag} rho {er:.3e} u {eu:.3e} (tol {tol})"
    assert_regions(rg, ug, ro, uo, o.n, tuple(o.params.bc_lo), tuple(o.params.bc_hi), tol, tag)
    return er, eu


TOL = {"fp64": 1e-11, "fp32": 1e-5}


LAYOUTS = [(2, 0, 1), (0, 1, 2)]  # (wall, span, flow): walls across z / across x

# storage and step pass: FP64 always takes the flat pass; FP32 runs the fused
# row pass (auto: momentum and step in one launch, where axis 2 is
# non-periodic), the row pass with a separate momentum kernel, and the flat pass
KERNELS = [("fp64", "auto"), ("fp32", "auto"), ("fp32", "rows"), ("fp32", "flat")]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("storage,kernel", KERNELS)
def test_plain_channel_1000_steps(storage, kernel, layout):
    """16x16x32 periodic channel (32 along the flow), static one-mode metric
    (5 %), walls, body force, tau = 0.8, rho = 1, u = 0, 1000 steps."""
    n = [0, 0, 0]
    n[layout[0]], n[layout[1]], n[layout[2]] = 16, 16, 32
    w = I.plain_fp64_channel(tuple(n), layout)
    g, o = make_pair(w, storage, step_kernel=kernel)
    g.init_equilibrium()
    o.init()
    rg, ug = g.moments()
    assert rel(rg, o.moments()[0]) < TOL[storage]  # rest at t = 0
    assert np.abs(ug).max() < (1e-12 if storage == "fp64" else 1e-6)
    g.step(1000)
    o.step(1000)
    compare(g, o, w["chart"].J9, TOL[storage], "t=1000")
    mo, mg = o.mass(), g.total_mass()
    assert abs(mg - mo) / mo < (1e-12 if storage == "fp64" else 1e-6)
    for side in (0, 1):
        fo = o.wall_force(layout[0], side, w["chart"].J9)
        fg = g.wall_force(layout[0], side)
        assert rel(fg, fo) < (1e-10 if storage == "fp64" else 1e-5)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("storage", ["fp64", "fp32"])
def test_ragged_inflow_outflow_moving_wall(storage, layout):
    """Odd sizes that leave ragged tiles, inflow/outflow along the flow axis,
    a moving wall, random initial density and velocity, a 4-mode tapered
    deformation."""
    n = [0, 0, 0]
    n[layout[0]], n[layout[1]], n[layout[2]] = 13, 37, 29
    n = tuple(n)
    dfm = I.fourier_deformation(n, 4, 0.06, seed=77, flow_periodic=False, kmax=2, lmax=1, layout=layout)
    ch = I.channel_chart(n, dfm, layout)
    rng = np.random.default_rng(5)
    nwall = I.face_nodes(n, layout[0], 1).size
    faces = {(layout[2], 0): I.inflow_profile(n, ch, 0.04, layout),
             (layout[0], 1): 0.01 * rng.standard_normal((3, nwall))}
    lo, hi = [P] * 3, [P] * 3
    lo[layout[0]] = hi[layout[0]] = W
    lo[layout[2]], hi[layout[2]] = IN, OUT
    fext = [1e-5, 0.0, 0.0]
    fext[layout[2]] = 2e-5
    w = dict(n=n, bc_lo=tuple(lo), bc_hi=tuple(hi), tau=0.7, fext=tuple(fext), chart=ch, faces=faces)
    g, o = make_pair(w, storage)
    N = int(np.prod(n))
    rho0 = 1 + 0.01 * rng.standard_normal(N)
    u0 = 0.02 * rng.standard_normal((3, N))
    g.init_equilibrium(rho0, u0)
    o.init(rho0, u0)
    g.step(150)
    o.step(150)
    compare(g, o, ch.J9, TOL[storage])


def test_walls_on_every_axis_edges_and_corners():
    """All six faces are walls (edges and corners take the wall rule with the
    diagonal inner node); one wall moves."""
    n = (35, 9, 7)
    dfm = I.fourier_deformation(n, 2, 0.04, seed=3, flow_periodic=False, kmax=1, lmax=1)
    ch = I.channel_chart(n, dfm)
    rng = np.random.default_rng(6)
    faces = {(2, 1): 0.02 * rng.standard_normal((3, 35 * 9))}
    w = dict(n=n, bc_lo=(W, W, W), bc_hi=(W, W, W), tau=0.9, fext=(0.0, 1e-5, 0.0), chart=ch, faces=faces)
    for storage in ("fp64", "fp32"):
        g, o = make_pair(w, storage)
        g.init_equilibrium()
        o.init()
        g.step(120)
        o.step(120)
        compare(g, o, ch.J9, TOL[storage], storage)
        for axis in range(3):
            for side in (0, 1):
                assert rel(g.wall_force(axis, side), o.wall_force(axis, side, ch.J9)) < 100 * TOL[storage]


@pytest.mark.parametrize("literal", [False, True])
def test_dynamic_metric_with_transform(literal):
    """Time-dependent deformation (dynamic channel generator at a small size):
    the metric and the distributions are re-transformed every 10 steps."""
    n = (9, 45, 17)
    w = I.dynamic_channel(n=n, seed=2000, n_modes=6, amp=0.06, tau=0.6, re=20.0, period=400.0, kmax=2,
                          lmax=1)
    for storage in ("fp64", "fp32"):
        g, o = make_pair(w, storage, literal)
        g.init_equilibrium()
        o.init()
        ch_old = w["chart"]
        for t in range(10, 110, 10):
            g.step(10)
            o.step(10)
            ch, faces = I.dynamic_channel_at(w, float(t))
            g.update_metric(ch.g6, ch.dg18, ch.J9)
            o.transform(ch.g6, ch.dg18, ch_old.J9, ch.J9)
            for (axis, side), u in faces.items():
                g.set_boundary_velocity(axis, side, u)
                o.set_face_velocity(axis, side, u)
            ch_old = ch
        g.step(5)
        o.step(5)
        compare(g, o, ch_old.J9, TOL[storage], storage)


@pytest.mark.parametrize("kernel", ["auto", "rows", "flat"])
@pytest.mark.parametrize("storage,tol", [("fp16", 3e-2), ("bf16", 1e-1)])
def test_reduced_precision_storage_error(storage, tol, kernel):
    """Weight-shifted FP16/BF16 storage with FP32 arithmetic, error vs the
    FP64 oracle on the plain channel after 1000 steps (stated bounds)."""
    w = I.plain_fp64_channel()
    g, o = make_pair(w, storage, step_kernel=kernel)
    g.init_equilibrium()
    o.init()
    g.step(1000)
    o.step(1000)
    rg, ug = g.moments(cartesian=True)
    ro, uo = o.moments(w["chart"].J9)
    er, eu = rel(rg, ro), rel(ug, uo)
    print(f"{storage}: rel L2 rho {er:.3e} u {eu:.3e}")
    assert er < 1e-3
    assert eu < tol


def test_flat_periodic_random_state_fp64():
    n = (5, 6, 7)
    w = dict(n=n, bc_lo=(P, P, P), bc_hi=(P, P, P), tau=0.55, fext=(1e-5, 2e-5, -1e-5), chart=I.flat_chart(n))
    g, o = make_pair(w, "fp64")
    rng = np.random.default_rng(8)
    N = int(np.prod(n))
    rho0 = 1 + 0.03 * rng.standard_normal(N)
    u0 = 0.05 * rng.standard_normal((3, N))
    g.init_equilibrium(rho0, u0)
    o.init(rho0, u0)
    g.step(200)
    o.step(200)
    compare(g, o, w["chart"].J9, 1e-12)
    assert abs(g.total_mass() - o.mass()) / o.mass() < 1e-13


def test_host_and_device_inputs_agree_and_state_roundtrip():
    import torch
    from paper_1803_07822_gb300.lattice import CurvedLattice
    w = I.plain_fp64_channel()
    ch = w["chart"]
    a = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    b = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    a.set_chart(ch)
    dev = lambda x: torch.as_tensor(x, device="cuda")
    b.set_metric(dev(ch.g6), dev(ch.dg18))
    b.set_jacobian(dev(ch.J9))
    a.init_equilibrium()
    b.init_equilibrium()
    a.step(20)
    b.step(20)
    ra, ua = a.moments()
    rb, ub = b.moments(host=False)
    assert np.array_equal(ra, rb.cpu().numpy()) and np.array_equal(ua, ub.cpu().numpy())
    snap = a.save_state()
    a.step(7)
    r1, u1 = a.moments()
    a.load_state(snap)
    a.step(7)
    r2, u2 = a.moments()
    assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
    assert a.check()


# Shapes for the row-staged step pass (FP32 storage, n0 a multiple of 4 and
# at most 256; a tile is floor(256 / n0) whole x-rows of one plane): a ragged
# last tile per plane, one 256-node row per tile, rows that straddle warps,
# walls across x (face lanes inside staged rows), periodic flow, and a
# lattice periodic on all three axes (every wrap of the row copies).
TILED = [
    ("ragged last tile", (20, 29, 13), (2, 0, 1), "inout"),
    ("one row per tile", (256, 24, 12), (2, 0, 1), "inout"),
    ("one row per tile, periodic flow", (256, 16, 10), (2, 0, 1), "periodic"),
    ("rows straddle warps", (100, 24, 10), (2, 0, 1), "periodic"),
    ("span-x two tiles", (64, 16, 9), (2, 0, 1), "inout"),
    ("walls across x", (32, 16, 40), (0, 1, 2), "inout"),
    ("periodic flow", (32, 32, 16), (2, 0, 1), "periodic"),
    ("periodic everywhere", (8, 6, 7), None, "torus"),
]


def smooth_wall_velocity(n, layout, amp=0.005):
    """A smooth contravariant velocity on the moving wall (face wall-axis, high)."""
    nodes = I.face_nodes(n, layout[0], 1)
    r = I.grid(n)
    p, s = r[layout[1]][nodes], r[layout[2]][nodes]
    u = np.zeros((3, nodes.size))
    u[layout[2]] = amp * np.cos(2 * np.pi * p / n[layout[1]]) * np.sin(np.pi * s / (n[layout[2]] - 1)) ** 2
    return u


def tiled_case(n, layout, kind):
    if kind == "torus":
        ch = I.flat_chart(n)
        return dict(n=n, bc_lo=(P, P, P), bc_hi=(P, P, P), tau=0.6, fext=(1e-5, -2e-5, 1e-5), chart=ch)
    if kind == "periodic":
        w = I.periodic_channel(n, 0.7, 0.04, 3, 0.05, 12, layout=layout)
        w["faces"] = {(layout[0], 1): smooth_wall_velocity(n, layout)}
        return w
    dfm = I.fourier_deformation(n, 4, 0.06, seed=13, flow_periodic=False, kmax=2, lmax=1, layout=layout)
    ch = I.channel_chart(n, dfm, layout)
    lo, hi = [P] * 3, [P] * 3
    lo[layout[0]] = hi[layout[0]] = W
    lo[layout[2]], hi[layout[2]] = IN, OUT
    return dict(n=n, bc_lo=tuple(lo), bc_hi=tuple(hi), tau=0.65, fext=(0.0, 0.0, 0.0), chart=ch,
                faces={(layout[2], 0): I.inflow_profile(n, ch, 0.04, layout),
                       (layout[0], 1): smooth_wall_velocity(n, layout)})


@pytest.mark.parametrize("kernel", ["auto", "rows", "flat"])
@pytest.mark.parametrize("name,n,layout,kind", TILED, ids=[t[0] for t in TILED])
def test_tiled_fp32(name, n, layout, kind, kernel):
    rng = np.random.default_rng(11)
    w = tiled_case(n, layout, kind)
    g, o = make_pair(w, "fp32", step_kernel=kernel)
    N = int(np.prod(n))
    rho0 = 1 + 0.005 * rng.standard_normal(N)
    u0 = 0.01 * rng.standard_normal((3, N))
    g.init_equilibrium(rho0, u0)
    o.init(rho0, u0)
    g.step(120)
    o.step(120)
    assert g.check()
    compare(g, o, w["chart"].J9, TOL["fp32"], name)


@pytest.mark.parametrize("kernel", ["auto", "rows"])
@pytest.mark.parametrize("name,n,layout,kind", TILED[:3], ids=[t[0] for t in TILED[:3]])
def test_row_staged_and_flat_passes_agree(name, n, layout, kind, kernel):
    """The step passes compute the same arithmetic per node (the fused pass
    forms rho u of face nodes in closed form from their inner nodes); after
    50 steps they agree to FP32 rounding."""
    w = tiled_case(n, layout, kind)
    a, _ = make_pair(w, "fp32", step_kernel=kernel)
    b, _ = make_pair(w, "fp32", step_kernel="flat")
    a.init_equilibrium()
    b.init_equilibrium()
    a.step(50)
    b.step(50)
    ra, ua = a.moments()
    rb, ub = b.moments()
    assert rel(ra, rb) < 1e-6 and rel(ua, ub) < 1e-5
