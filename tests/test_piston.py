"""The coupled loop with a prescribed-motion shell: a rigid piston pressing a
closed box by 0.2 % of its volume (the piston test of the coupled system).
The paper's invariants -- mass conserved (to 0.1 %), the lateral momenta
negligible against the normal one, the impulse on the piston equal to
pressure x area x time -- on the oracle loop (CPU) and on the library's loop
(GPU), and the library's loop against the oracle's step by step."""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300.coupling import THETA, piston_chart, piston_law

W = 2  # the wall-normal axis of the default layout


def oracle_piston(n, steps, T, amp, sample, tau=0.8):
    """The same loop as coupling.run_piston on the oracle."""
    H = n[W] - 1
    o = oracle.Lattice(n, (0, 0, 1), (0, 0, 1), tau=tau)
    ch = piston_chart(n, 0.0)
    o.set_metric(ch.g6, ch.dg18)
    o.init()
    nf = o.face_shape(W)
    out = {k: [] for k in ("mass", "momentum", "force", "impulse", "impulse_pA")}
    imp, imp_pa = np.zeros(3), 0.0
    for t in range(steps):
        d, dd = piston_law(float(t), T, amp, H)
        if t > 0:
            cn = piston_chart(n, d)
            o.transform(cn.g6, cn.dg18, ch.J9, cn.J9)
            ch = cn
        u3 = np.zeros((3, nf))
        u3[W] = dd / (1.0 + d / H)
        o.set_face_velocity(W, 1, u3)
        o.step(1)
        F = o.wall_force(W, 1, ch.J9)
        sg = ch.J9[8] * ch.J9[0] * ch.J9[4]
        m = o.mass()
        imp += F
        imp_pa += m / sg.sum() * THETA * nf
        if t % sample == 0 or t == steps - 1:
            r, v = o.moments(ch.J9)
            out["mass"].append(m)
            out["momentum"].append((sg * r * v).sum(axis=1))
            out["force"].append(F)
            out["impulse"].append(imp.copy())
            out["impulse_pA"].append(imp_pa)
    return {k: np.array(v) for k, v in out.items()}


def check_invariants(r, tol_mass):
    m = r["mass"]
    assert np.abs(m / m[0] - 1).max() < tol_mass
    P = r["momentum"]
    assert np.abs(P[:, :2]).max() < 1e-6 * np.abs(P[:, 2]).max()
    assert np.abs(P[:, 2]).max() > 0
    assert np.abs(r["impulse"][:, 2] / r["impulse_pA"] - 1).max() < 1e-3


def test_oracle_piston_invariants():
    r = oracle_piston((8, 8, 16), 500, 400, 0.002, 50)
    check_invariants(r, 1e-5)


@pytest.mark.gpu
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_piston_loop_matches_oracle(storage, tol):
    from paper_1803_07822_gb300.coupling import run_piston
    n, steps, T, amp, sample = (8, 8, 16), 160, 100, 0.01, 20
    g = run_piston(n, steps, T, amp, storage=storage, sample=sample)
    o = oracle_piston(n, steps, T, amp, sample)
    for k in ("mass", "force", "impulse"):
        err = np.abs(g[k] - o[k]).max() / np.abs(o[k]).max()
        assert err < tol, (k, err)
    err = np.abs(g["momentum"][:, 2] - o["momentum"][:, 2]).max() / np.abs(o["momentum"][:, 2]).max()
    assert err < 10 * tol, err


@pytest.mark.gpu
def test_piston_invariants_on_the_gpu():
    from paper_1803_07822_gb300.coupling import run_piston
    r = run_piston((32, 32, 64), 3000, 2000, 0.002, storage="fp32", sample=100)
    dv = 1 - r["volume"][-1] / r["volume"][0]
    print(f"\npiston 32x32x64, volume change {dv:.4%}: mass drift {np.abs(r['mass'] / r['mass'][0] - 1).max():.2e}, "
          f"|P_xy|/|P_z| {np.abs(r['momentum'][:, :2]).max() / np.abs(r['momentum'][:, 2]).max():.1e}, "
          f"impulse / (p A t) - 1 {np.abs(r['impulse'][:, 2] / r['impulse_pA'] - 1).max():.1e}")
    assert 0.0019 < dv < 0.0021
    check_invariants(r, 1e-3)
