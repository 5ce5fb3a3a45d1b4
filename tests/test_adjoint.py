"""Adjoint: gradient of the streamwise force on the deformed wall after 200
steps from rest with respect to the Fourier coefficients of the wall
deformation, through the library's checkpointed adjoint (every 20 steps) and
the torch chart map, against central finite differences (h = 1e-4) of the
FP64 oracle (small channel) and of the FP64 GPU forward (adjoint-form
channel 64 x 128 x 64, 32 coefficients)."""
import time

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

STEPS, EVERY, H_FD = 200, 20, 1e-4


def case(n, kmax, lmax, seed, tau=0.8, shrink=1.0):
    """d = H / (shrink sqrt(M)) sum_m c_m cos(2 pi k_m s / L_s + 2 pi l_m p / L_p), c_m ~ N(0, 0.02)."""
    return I.adjoint_channel(n, kmax, lmax, seed, tau, shrink)


def e_flow(w):
    e = [0.0, 0.0, 0.0]
    e[w["layout"][2]] = 1.0
    return e


def adjoint_grad(w, storage):
    import torch
    from paper_1803_07822_gb300.adjoint import chart_from_coeffs, wall_force_objective
    from paper_1803_07822_gb300.lattice import CurvedLattice
    lat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage=storage,
                        step_kernel="flat")
    c = torch.tensor(w["c"], dtype=torch.float64, device="cuda", requires_grad=True)
    g6, dg18, J9 = chart_from_coeffs(c, w["n"], w["modes"], w["scale"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = wall_force_objective(lat, g6, dg18, J9, STEPS, EVERY, axis=w["layout"][0], side=1, e3=e_flow(w))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return float(J), c.grad.cpu().numpy(), (t2 - t1) / (t1 - t0)


def oracle_objective(w, c):
    ch = I.periodic_channel(w["n"], w["tau"], 0.05, len(c), w["scale"], 0, modes=w["modes"], coeffs=c)["chart"]
    o = oracle.Lattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"])
    o.set_metric(ch.g6, ch.dg18)
    o.init()
    o.step(STEPS)
    return float(np.dot(e_flow(w), o.wall_force(w["layout"][0], 1, ch.J9)))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_torch_chart_matches_the_generator():
    torch = pytest.importorskip("torch")
    from paper_1803_07822_gb300.adjoint import chart_from_coeffs
    w = case((12, 20, 10), 2, 1, 7)
    ch = I.periodic_channel(w["n"], w["tau"], 0.05, len(w["c"]), w["scale"], 0, modes=w["modes"], coeffs=w["c"])
    g6, dg18, J9 = chart_from_coeffs(torch.tensor(w["c"], dtype=torch.float64), w["n"], w["modes"], w["scale"])
    for a, b in ((g6, ch["chart"].g6), (dg18, ch["chart"].dg18), (J9, ch["chart"].J9)):
        assert np.abs(a.numpy() - b).max() < 1e-13


@pytest.fixture(scope="module")
def small():
    """16 x 32 x 16 channel (32 along the flow), 8 coefficients, and the
    central differences of the FP64 oracle's objective."""
    w = case((16, 32, 16), 4, 1, 5000)
    fd = np.zeros(len(w["c"]))
    for m in range(len(w["c"])):
        cp, cm = w["c"].copy(), w["c"].copy()
        cp[m] += H_FD
        cm[m] -= H_FD
        fd[m] = (oracle_objective(w, cp) - oracle_objective(w, cm)) / (2 * H_FD)
    return w, fd


@pytest.mark.gpu
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-4), ("fp32", 1e-2)])
def test_adjoint_matches_oracle_finite_differences(small, storage, tol):
    w, fd = small
    J, g, ratio = adjoint_grad(w, storage)
    J0 = oracle_objective(w, w["c"])
    assert abs(J - J0) <= 1e-9 * max(1.0, abs(J0)) if storage == "fp64" else abs(J - J0) <= 1e-4 * abs(J0)
    err = rel(g, fd)
    print(f"\n{storage}: objective {J:.6e}, gradient rel err vs oracle FD {err:.3e}, adjoint/forward time {ratio:.1f}")
    assert err < tol


@pytest.mark.gpu
def test_adjoint_form_channel_against_gpu_finite_differences():
    """The adjoint-form channel 64 x 128 x 64 (span, flow, wall), 32
    coefficients from N(0, 0.02), k in 1..8 along the flow, l in 0..3 across,
    d = H / (4 sqrt(32)) sum c_m phi_m (largest wall slope 0.25: with H /
    sqrt(32) the slope reaches 1.0 and the method is unstable): FP32 adjoint
    against central differences of the FP64 GPU forward on three coefficients."""
    import torch
    from paper_1803_07822_gb300.adjoint import chart_from_coeffs
    from paper_1803_07822_gb300.lattice import CurvedLattice
    w = case((64, 128, 64), 8, 3, 5000, shrink=4.0)
    J, g, ratio = adjoint_grad(w, "fp32")
    lat = CurvedLattice(w["n"], w["bc_lo"], w["bc_hi"], tau=w["tau"], fext=w["fext"], storage="fp64",
                        step_kernel="flat")

    def objective(c):
        g6, dg18, J9 = chart_from_coeffs(torch.tensor(c, dtype=torch.float64, device="cuda"), w["n"], w["modes"],
                                         w["scale"])
        lat.set_metric(g6, dg18)
        lat.set_jacobian(J9)
        lat.init_equilibrium()
        lat.step(STEPS)
        return float(np.dot(e_flow(w), lat.wall_force(w["layout"][0], 1)))

    picks = [0, 9, 27]
    fd = []
    for m in picks:
        cp, cm = w["c"].copy(), w["c"].copy()
        cp[m] += H_FD
        cm[m] -= H_FD
        fd.append((objective(cp) - objective(cm)) / (2 * H_FD))
    err = rel(g[picks], fd)
    print(f"\n64x128x64: gradient rel err (3 coefficients) {err:.3e}, adjoint/forward time {ratio:.1f}")
    assert err < 1e-2
