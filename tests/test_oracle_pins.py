"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against a property it does not compute itself:
quadrature identities of the lattice (App. B), the textbook flat-space
equilibrium, closed forms of the Christoffel symbols of a chart of flat space
(App. A), metric compatibility, and the continuum balances that the forcing
moments A and B were built to satisfy (App. C).
"""
import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

CS2 = 1.0 / 3.0


def test_d3q19_set_and_isotropy():
    c, w = oracle.lattice()
    assert c.shape == (19, 3)
    # 1 rest, 6 faces (|c|^2 = 1), 12 edges (|c|^2 = 2); every c has its opposite
    n2 = (c * c).sum(1)
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert len({tuple(v) for v in c}) == 19
    for v in c:
        assert any((u == -v).all() for u in c)
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("l,li->i", w, c)).max() < 1e-15
    assert np.allclose(np.einsum("l,li,lj->ij", w, c, c), CS2 * d, atol=1e-15)
    assert np.abs(np.einsum("l,li,lj,lk->ijk", w, c, c, c)).max() < 1e-15
    four = np.einsum("l,li,lj,lk,lm->ijkm", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ij,km->ijkm", d, d) + np.einsum("ik,jm->ijkm", d, d)
                      + np.einsum("im,jk->ijkm", d, d))
    assert np.allclose(four, iso, atol=1e-15)


def test_equilibrium_moments_any_metric():
    """sum f^eq sqrt g = rho, sum f^eq c sqrt g = rho u,
    sum f^eq c c sqrt g = rho (theta g^-1 + u u)   (App. B)."""
    c, _ = oracle.lattice()
    rng = np.random.default_rng(1)
    for _ in range(20):
        g = I.random_spd_metric(rng)
        gi = np.linalg.inv(g)
        sg = np.sqrt(np.linalg.det(g))
        rho = 1.0 + 0.2 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        theta = CS2 * (1.0 + 0.1 * rng.standard_normal())
        f = oracle.feq(rho, rho * u, gi.ravel(), sg, theta)
        assert abs((f * sg).sum() - rho) < 1e-14
        assert np.allclose(np.einsum("l,li->i", f * sg, c), rho * u, atol=1e-15)
        Pi = np.einsum("l,li,lj->ij", f * sg, c, c)
        assert np.allclose(Pi, rho * (theta * gi + np.outer(u, u)), atol=1e-14)


def test_equilibrium_flat_is_textbook():
    """At g = delta, theta = c_s^2 the expansion is the standard D3Q19 BGK
    equilibrium w rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    c, w = oracle.lattice()
    rng = np.random.default_rng(2)
    for _ in range(10):
        rho = 1.0 + 0.1 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        f = oracle.feq(rho, rho * u, np.eye(3).ravel(), 1.0)
        cu = c @ u
        ref = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u @ u))
        assert np.allclose(f, ref, atol=1e-15, rtol=0)


def test_forcing_recomposition_moments():
    """sum F sqrt g = A, sum F c sqrt g = B, sum F c c sqrt g = C (Eqs. forcing-A/B/C)."""
    c, _ = oracle.lattice()
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.standard_normal()
        B = rng.standard_normal(3)
        C = rng.standard_normal((3, 3))
        C = C + C.T
        sg = 0.8 + 0.4 * rng.random()
        F = oracle.forcing_recompose(A, B, C.ravel(), sg)
        assert abs((F * sg).sum() - A) < 1e-14
        assert np.allclose(np.einsum("l,li->i", F * sg, c), B, atol=1e-14)
        assert np.allclose(np.einsum("l,li,lj->ij", F * sg, c, c), C, atol=1e-14)


def _charts():
    n = (9, 8, 12)
    dfm = I.fourier_deformation(n, 4, 0.08, seed=11, flow_periodic=True)
    yield I.channel_chart(n, dfm)
    dfm = I.fourier_deformation(n, 4, 0.08, seed=12, flow_periodic=False)
    yield I.channel_chart(n, dfm)
    yield I.reparam_chart(n, 0.1)
    yield I.annulus_chart(n, 6.0)  # polar coordinates: Gamma^r_tt and Gamma^t_rt nonzero


@pytest.mark.parametrize("chart", list(_charts()))
def test_geometry_closed_forms(chart):
    """g g^-1 = I; sqrt g = det J; Gamma^i_jk = (J^-1)^i_a d_j d_k h^a for a
    chart of flat space; metric compatibility d_k g_ij = Gamma^l_ki g_lj +
    Gamma^l_kj g_il (App. A)."""
    n, N = chart.n, chart.N
    sg, gi, gam = oracle.geometry(n, chart.g6, chart.dg18)
    g = np.zeros((3, 3, N))
    for m, (i, j) in enumerate(I.SYM):
        g[i, j] = g[j, i] = chart.g6[m]
    giv = gi.reshape(3, 3, N)
    assert np.abs(np.einsum("ijn,jkn->ikn", g, giv) - np.eye(3)[:, :, None]).max() < 1e-13
    J = chart.J9.reshape(3, 3, N)
    assert np.abs(sg - np.linalg.det(np.moveaxis(J, 2, 0))).max() < 1e-13
    Jinv = np.linalg.inv(np.moveaxis(J, 2, 0))  # [N, i, a]
    Hs = chart.hess.reshape(3, 3, 3, N)
    closed = np.einsum("nia,ajkn->ijkn", Jinv, Hs)
    assert np.abs(gam.reshape(3, 3, 3, N) - closed).max() < 1e-13
    G = gam.reshape(3, 3, 3, N)
    dg = np.zeros((3, 3, 3, N))
    for k in range(3):
        for m, (i, j) in enumerate(I.SYM):
            dg[k, i, j] = dg[k, j, i] = chart.dg18[k * 6 + m]
    comp = np.einsum("lkin,ljn->kijn", G, g) + np.einsum("lkjn,iln->kijn", G, g)
    assert np.abs(comp - dg).max() < 1e-13


def test_sqrtg_derivative_identity_converges():
    """d_i sqrt g = Gamma^j_ij sqrt g (App. C): central differences of the
    oracle's sqrt g along the flow axis converge to it at second order."""
    errs = []
    for n2 in (32, 64):
        n = (5, 4, n2)
        lay = (0, 1, 2)  # flow along axis 2
        dfm = I.fourier_deformation(n, 3, 0.08, seed=5, flow_periodic=True, kmax=2, layout=lay)
        ch = I.channel_chart(n, dfm, lay)
        sg, _, gam = oracle.geometry(n, ch.g6, ch.dg18)
        s3 = sg.reshape(n2, 4, 5)
        G = gam.reshape(3, 3, 3, -1)
        gc2 = (G[0, 2, 0] + G[1, 2, 1] + G[2, 2, 2]).reshape(n2, 4, 5) * s3
        fd = (np.roll(s3, -1, 0) - np.roll(s3, 1, 0)) / 2.0
        errs.append(np.abs(fd - gc2).max())
    assert errs[1] < errs[0] / 3.2


def test_forcing_A_B_balance_continuum():
    """A and B are the sources that turn the lattice balances into covariant
    ones (App. C):  A = dbar_i j^i - nabla_i j^i with nabla_i j^i =
    (1/sqrt g) d_i (sqrt g j^i) (App. A divergence), and at rest
    (T = rho theta g^-1) B^i = dbar_j (rho theta g^ij), where d_k g^ij =
    -g^il d_k g_lm g^mj and d_i sqrt g = 1/2 sqrt g g^jk d_i g_jk are taken
    from the metric derivatives alone."""
    rng = np.random.default_rng(7)
    for _ in range(10):
        g = I.random_spd_metric(rng)
        gi = np.linalg.inv(g)
        dg = rng.standard_normal((3, 3, 3)) * 0.1
        dg = dg + dg.transpose(0, 2, 1)  # d_k g_ij symmetric in ij
        g6 = np.array([g[i, j] for i, j in I.SYM])[:, None]
        dg18 = np.array([dg[k, i, j] for k in range(3) for i, j in I.SYM])[:, None]
        sg, giv, gam = oracle.geometry((1, 1, 1), g6, dg18)
        gam27 = gam[:, 0]
        theta = CS2
        rho = 1.0 + 0.1 * rng.standard_normal()
        j = 0.1 * rng.standard_normal(3)
        Dj = rng.standard_normal((3, 3)) * 0.01
        # continuity source
        A, _, _ = oracle.forcing_moments(j, (rho * theta * gi).ravel(), Dj.ravel(), gi.ravel(),
                                         gam27, theta)
        dsg_over_sg = 0.5 * np.einsum("jk,ijk->i", gi, dg)
        G = gam27.reshape(3, 3, 3)
        trace = np.einsum("jij->i", G)
        divbar = np.trace(Dj) - trace @ j
        divcov = np.trace(Dj) + dsg_over_sg @ j
        assert abs(A - (divbar - divcov)) < 1e-14
        # rest momentum source
        T = rho * theta * gi
        _, B, _ = oracle.forcing_moments(np.zeros(3), T.ravel(), np.zeros(9), gi.ravel(), gam27,
                                         theta)
        dginv = -np.einsum("il,klm,mj->kij", gi, dg, gi)  # d_k g^ij
        expect = rho * theta * (np.einsum("jij->i", dginv) - np.einsum("j,ij->i", trace, gi))
        assert np.allclose(B, expect, atol=1e-14)


def test_forcing_flat_reduces_to_body_force():
    """At g = delta, Gamma = 0 and theta = c_s^2: A = 0, C = 0, B = F_ext for
    any velocity gradient, so F_l = w_l c_l . F_ext / c_s^2."""
    c, w = oracle.lattice()
    rng = np.random.default_rng(9)
    fext = rng.standard_normal(3)
    A, B, C = oracle.forcing_moments(rng.standard_normal(3), rng.standard_normal(9),
                                     rng.standard_normal(9), np.eye(3).ravel(), np.zeros(27),
                                     CS2, fext)
    assert abs(A) < 1e-15 and np.abs(C).max() < 1e-14 and np.allclose(B, fext, atol=1e-15)
    F = oracle.forcing_recompose(A, B, C, 1.0)
    assert np.allclose(F, w * (c @ fext) / CS2, atol=1e-14)


def test_annulus_chart_derivatives():
    """The polar chart's J and second derivatives are those of h(x, y, z) =
    ((r0 + x) cos(y/r0), (r0 + x) sin(y/r0), z): central differences of h
    (step 1e-4) at the nodes."""
    n, r0, e = (5, 7, 3), 6.0, 1e-4
    ch = I.annulus_chart(n, r0)
    x, y, z = I.grid(n)

    def h(x, y, z):
        return np.stack([(r0 + x) * np.cos(y / r0), (r0 + x) * np.sin(y / r0), z])

    X = [x, y, z]
    for i in range(3):
        d = [0.0, 0.0, 0.0]
        d[i] = e
        col = (h(*(X[k] + d[k] for k in range(3))) - h(*(X[k] - d[k] for k in range(3)))) / (2 * e)
        for a in range(3):
            assert np.abs(ch.J9[a * 3 + i] - col[a]).max() < 1e-8
            for j in range(3):
                dj = [0.0, 0.0, 0.0]
                dj[j] = e
                Jp = (h(*(X[k] + d[k] + dj[k] for k in range(3))) - h(*(X[k] - d[k] + dj[k] for k in range(3))))
                Jm = (h(*(X[k] + d[k] - dj[k] for k in range(3))) - h(*(X[k] - d[k] - dj[k] for k in range(3))))
                second = (Jp - Jm) / (4 * e * e)
                assert np.abs(ch.hess[a * 9 + i * 3 + j] - second[a]).max() < 1e-5


@pytest.mark.parametrize("chart", list(_charts()))
def test_forcing_C_parallel_field_has_no_theta_part(chart):
    """A uniform Cartesian flow V is a parallel field of flat space, so its
    covariant derivative vanishes in every chart: with j^i = (J^-1)^i_a V^a,
    d_k j^i = -(J^-1)^i_b d_k J^b_m j^m cancels Gamma^i_kl j^l exactly
    (App. A).  The theta part of C^ij (Eq. forcing-C) is built from nabla_k j^i
    alone, so C does not depend on theta for such a field.  Dropping the
    Gamma^i_kl rho u^l term, or transposing its indices, leaves the partial
    derivative in its place and C then moves with theta."""
    n, N = chart.n, chart.N
    sg, gi, gam = oracle.geometry(n, chart.g6, chart.dg18)
    J = np.moveaxis(chart.J9.reshape(3, 3, N), 2, 0)   # [n, a, i]
    Jinv = np.linalg.inv(J)                             # [n, i, a]
    dJ = np.moveaxis(chart.hess.reshape(3, 3, 3, N), 3, 0)  # [n, b, m, k] = d_k J^b_m
    rng = np.random.default_rng(21)
    worst, scale = 0.0, 0.0
    for v in rng.choice(N, size=12, replace=False):
        V = 0.05 * rng.standard_normal(3)
        rho = 1.0 + 0.05 * rng.standard_normal()
        j = rho * Jinv[v] @ V
        Dj = -np.einsum("ib,bmk,m->ki", Jinv[v], dJ[v], j)  # [k, i] = d_k j^i
        T = rng.standard_normal((3, 3))
        T = T + T.T
        C = []
        for theta in (CS2, 0.25):
            _, _, c9 = oracle.forcing_moments(j, T.ravel(), Dj.ravel(), gi[:, v], gam[:, v], theta)
            C.append(c9)
        worst = max(worst, np.abs(C[0] - C[1]).max())
        # what the theta part amounts to when the Christoffel term is left out
        C0 = [oracle.forcing_moments(j, T.ravel(), Dj.ravel(), gi[:, v], np.zeros(27), th)[2]
              for th in (CS2, 0.25)]
        scale = max(scale, np.abs(C0[0] - C0[1]).max())
    assert worst < 1e-15 + 1e-12 * scale, (worst, scale)
    if np.abs(gam).max() > 1e-3:
        assert scale > 1e-5  # the pin has teeth on this chart
