"""Pins of the oracle's isotropic lattice derivatives (App. D): exactness on
polynomials up to the stencil's order (faces, edges and corners included),
inexactness one degree above, and the convergence slopes -2 / -4 of the
gradient of a periodic field and of the channel metric against its analytic
derivative -- the paper's derivative convergence study."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1803_07822_gb300 import inputs as I

WALLS = (1, 1, 1)


def coords(n):
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return x.ravel().astype(float), y.ravel().astype(float), z.ravel().astype(float)


def random_poly(deg, seed):
    """{(p, q, r): a} with p + q + r <= deg, every monomial present."""
    rng = np.random.default_rng(seed)
    return {e: rng.normal() for e in itertools.product(range(deg + 1), repeat=3) if sum(e) <= deg}


def poly_eval(P, x, y, z, d=None):
    """The polynomial, or its derivative along axis d, from the monomials."""
    out = np.zeros_like(x)
    for (p, q, r), a in P.items():
        e = [p, q, r]
        c = a
        if d is not None:
            if e[d] == 0:
                continue
            c = a * e[d]
            e[d] -= 1
        out += c * x ** e[0] * y ** e[1] * z ** e[2]
    return out


@pytest.mark.parametrize("order", [2, 4])
def test_exact_on_polynomials_up_to_the_order(order):
    n = (7, 8, 9)
    x, y, z = coords(n)
    s = 0.1  # keep the monomials of order 1
    P = random_poly(order, 11 + order)
    f = poly_eval(P, s * x, s * y, s * z)
    g = oracle.lattice_gradient(n, f[None], order, bc_lo=WALLS)
    for d in range(3):
        ref = s * poly_eval(P, s * x, s * y, s * z, d)
        assert np.abs(g[d, 0] - ref).max() < 1e-11 * max(1.0, np.abs(ref).max()), d


@pytest.mark.parametrize("order", [2, 4])
def test_not_exact_one_degree_higher(order):
    n = (9, 9, 9)
    x, y, z = coords(n)
    f = (0.1 * x) ** (order + 1) + (0.1 * y) ** (order + 1)
    g = oracle.lattice_gradient(n, f[None], order, bc_lo=WALLS)
    ref = 0.1 * (order + 1) * (0.1 * x) ** order
    assert np.abs(g[0, 0] - ref).max() > 1e-6


@pytest.mark.parametrize("order", [2, 4])
def test_laplacian_exact_up_to_the_ghost_degree(order):
    """Exact on cubics inside; at the faces up to the continuation's degree."""
    n = (7, 8, 6)
    x, y, z = coords(n)
    P = random_poly(min(3, order), 21)
    s = 0.2
    f = poly_eval(P, s * x, s * y, s * z)
    lap = oracle.lattice_laplacian(n, f[None], order, bc_lo=WALLS)[0]
    ref = np.zeros_like(x)
    for (p, q, r), a in P.items():  # sum of second derivatives, monomial by monomial
        e = [p, q, r]
        for d in range(3):
            if e[d] >= 2:
                ee = list(e)
                ee[d] -= 2
                ref += s * s * a * e[d] * (e[d] - 1) * (s * x) ** ee[0] * (s * y) ** ee[1] * (s * z) ** ee[2]
    assert np.abs(lap - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


def slope(ms, errs):
    return np.polyfit(np.log(ms), np.log(errs), 1)[0]


@pytest.mark.parametrize("order,expect", [(2, -2.0), (4, -4.0)])
def test_convergence_periodic_field(order, expect):
    ms, errs = [16, 24, 32, 48], []
    for m in ms:
        n = (m, m, m)
        x, y, z = coords(n)
        k = 2 * np.pi / m
        f = np.sin(k * x + 0.3) * np.cos(2 * k * y) + np.sin(k * z)
        g = oracle.lattice_gradient(n, f[None], order)
        ref = np.stack([k * np.cos(k * x + 0.3) * np.cos(2 * k * y),
                        -2 * k * np.sin(k * x + 0.3) * np.sin(2 * k * y), k * np.cos(k * z)])
        errs.append(np.linalg.norm(g[:, 0] - ref) / np.linalg.norm(ref))
    assert abs(slope(ms, errs) - expect) < 0.2, (errs, slope(ms, errs))


@pytest.mark.parametrize("order,expect", [(2, -2.0), (4, -4.0)])
def test_convergence_of_the_channel_metric_derivative(order, expect):
    """Relative error of d_k g_ij from the lattice stencil against the chart's
    analytic derivative, walls across the wall axis, periodic span and flow,
    one oblique mode of 5 % of the height at every resolution."""
    ms, errs = [12, 16, 24, 32], []
    for m in ms:
        n = (m, 2 * m, m)
        w = I.periodic_channel(n, 0.8, 0.05, 1, 0.05, 0, modes=([1], [1], [0.3]), coeffs=[1.0])
        ch = w["chart"]
        g = oracle.lattice_gradient(n, ch.g6, order, bc_lo=w["bc_lo"], bc_hi=w["bc_hi"])
        errs.append(np.linalg.norm(g.reshape(18, -1) - ch.dg18) / np.linalg.norm(ch.dg18))
    assert abs(slope(ms, errs) - expect) < 0.2, (errs, slope(ms, errs))
