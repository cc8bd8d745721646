"""Pins of the oracle's velocity medium and Hamiltonian against independent facts.

The medium is the tensor-product cubic B-spline of the velocity samples (the
paper does not say how c is interpolated; the ray and dynamic-ray equations,
Eqs. characline, dzQ and dzP, need c, grad c and the Hessian of c, so a C^2
spline is the reading taken).
"""

import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_beta3_matches_scipy_basis_element():
    # library routine: scipy's cardinal cubic B-spline on knots -2..2 and its derivatives
    from scipy.interpolate import BSpline

    b = BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    n = 16
    h = 0.37
    g = O.Grid((n,), (h,), (0.0,), (False,))
    coef = np.zeros(n)
    i0 = 7
    coef[i0] = 1.0
    t = np.linspace(-1.97, 1.97, 157)
    t = t[np.abs(np.abs(t) - 1.0) > 1e-9]  # third derivative jumps at the knots
    t = t[np.abs(t) > 1e-9]
    x = (i0 + t) * h
    c, gr, hs, d3 = O.medium_eval(g, coef, x[:, None], order=3)
    np.testing.assert_allclose(c, b(t), rtol=0, atol=1e-15)
    np.testing.assert_allclose(gr[:, 0], b.derivative(1)(t) / h, rtol=0, atol=1e-13)
    np.testing.assert_allclose(hs[:, 0, 0], b.derivative(2)(t) / h ** 2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(d3[:, 0, 0, 0], b.derivative(3)(t) / h ** 3, rtol=0, atol=1e-11)


def test_spline_reproduces_linear_and_quadratic_2d():
    # cubic B-splines reproduce linear functions exactly; x^2 comes back as x^2 + h^2/3
    # (the variance of the cubic B-spline is 1/3) -- checked away from the clamped edges.
    n = (24, 20)
    h = (0.1, 0.07)
    o = (-0.3, 0.2)
    g = O.Grid(n, h, o, (False, False))
    xs = [o[k] + h[k] * np.arange(n[k]) for k in range(2)]
    X, Z = np.meshgrid(*xs, indexing="ij")
    rng = np.random.default_rng(0)
    pts = np.stack([rng.uniform(o[0] + 3 * h[0], o[0] + (n[0] - 4) * h[0], 50),
                    rng.uniform(o[1] + 3 * h[1], o[1] + (n[1] - 4) * h[1], 50)], axis=1)
    lin = 1.3 - 0.4 * X + 2.1 * Z
    c, gr, hs, _ = O.medium_eval(g, lin, pts)
    np.testing.assert_allclose(c, 1.3 - 0.4 * pts[:, 0] + 2.1 * pts[:, 1], atol=1e-13)
    np.testing.assert_allclose(gr, np.broadcast_to([-0.4, 2.1], gr.shape), atol=1e-12)
    np.testing.assert_allclose(hs, 0.0, atol=1e-10)
    quad = X ** 2
    c, gr, hs, _ = O.medium_eval(g, quad, pts)
    np.testing.assert_allclose(c, pts[:, 0] ** 2 + h[0] ** 2 / 3.0, atol=1e-13)
    np.testing.assert_allclose(gr[:, 0], 2 * pts[:, 0], atol=1e-12)
    np.testing.assert_allclose(hs[:, 0, 0], 2.0, atol=1e-10)
    np.testing.assert_allclose(hs[:, 1, 1], 0.0, atol=1e-10)


def test_spline_periodic_wraps():
    n = 12
    h = 1.0 / n
    g = O.Grid((n,), (h,), (0.0,), (True,))
    coef = np.cos(2 * np.pi * np.arange(n) * h)
    x = np.array([[0.013], [0.513], [0.987]])
    c1, g1, _, _ = O.medium_eval(g, coef, x)
    c2, g2, _, _ = O.medium_eval(g, coef, x + 1.0)
    c3, g3, _, _ = O.medium_eval(g, coef, x - 1.0)
    np.testing.assert_allclose(c1, c2, atol=1e-14)
    np.testing.assert_allclose(c1, c3, atol=1e-14)
    # at the knots the spline of a sampled sinusoid is the sinusoid scaled by
    # beta3(0) + 2 beta3(1) cos(2 pi h) = (2 + cos(2 pi h))/3
    lam = (2.0 + math.cos(2 * math.pi * h)) / 3.0
    xk = (np.arange(n) * h)[:, None]
    ck, _, _, _ = O.medium_eval(g, coef, xk)
    np.testing.assert_allclose(ck, lam * np.cos(2 * np.pi * xk[:, 0]), atol=1e-14)


def _smooth_field(n, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(n)
    from scipy.ndimage import gaussian_filter

    return 2.0 + 0.3 * gaussian_filter(f, 2.0, mode="wrap")


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_spline_derivatives_match_finite_differences(dim):
    n = (14, 12, 10)[:dim]
    h = (0.11, 0.09, 0.13)[:dim]
    o = (0.5, -0.2, 0.1)[:dim]
    g = O.Grid(n, h, o, (False,) * dim)
    coef = _smooth_field(n, 1)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(o[k] + 2 * h[k], o[k] + (n[k] - 3) * h[k], 20)
                    for k in range(dim)], axis=1)
    c, gr, hs, d3 = O.medium_eval(g, coef, pts, order=3)
    step = 1e-5
    for k in range(dim):
        e = np.zeros(dim)
        e[k] = step
        cp, gp, hp, _ = O.medium_eval(g, coef, pts + e, order=2)
        cm, gm, hm, _ = O.medium_eval(g, coef, pts - e, order=2)
        np.testing.assert_allclose((cp - cm) / (2 * step), gr[:, k], atol=1e-7)
        np.testing.assert_allclose((gp - gm) / (2 * step), hs[:, k, :], atol=1e-6)
        np.testing.assert_allclose((hp - hm) / (2 * step), d3[:, k, :, :], atol=1e-4)
    # symmetry of the Hessian
    np.testing.assert_allclose(hs, np.swapaxes(hs, 1, 2), atol=1e-12)


@pytest.mark.parametrize("sigma", [1, -1])
def test_hamiltonian_derivatives_match_finite_differences(sigma):
    # H = sigma c(Q)|P| (Eq. hamiltonian); every written-out derivative is checked
    # against central differences of H or of its first derivatives.
    dim = 2
    n = (16, 14)
    h = (0.1, 0.1)
    o = (0.0, 0.0)
    g = O.Grid(n, h, o, (False, False))
    coef = _smooth_field(n, 3)
    Q = np.array([0.73, 0.61])
    P = np.array([0.8, -0.45])
    ref = O.hamiltonian(g, coef, sigma, Q, P)
    c, gr, hs, _ = O.medium_eval(g, coef, Q[None])
    assert abs(ref["H"] - sigma * c[0] * np.linalg.norm(P)) < 1e-14
    step = 1e-6
    for k in range(dim):
        e = np.zeros(dim)
        e[k] = step
        Hq = (O.hamiltonian(g, coef, sigma, Q + e, P)["H"] - O.hamiltonian(g, coef, sigma, Q - e, P)["H"]) / (2 * step)
        Hp = (O.hamiltonian(g, coef, sigma, Q, P + e)["H"] - O.hamiltonian(g, coef, sigma, Q, P - e)["H"]) / (2 * step)
        assert abs(Hq - ref["dHdQ"][k]) < 1e-7
        assert abs(Hp - ref["dHdP"][k]) < 1e-7
        qp, qm = O.hamiltonian(g, coef, sigma, Q + e, P), O.hamiltonian(g, coef, sigma, Q - e, P)
        pp, pm = O.hamiltonian(g, coef, sigma, Q, P + e), O.hamiltonian(g, coef, sigma, Q, P - e)
        # row k of d2H/dQ_k dQ_l and d2H/dQ_k dP_l
        np.testing.assert_allclose((qp["dHdQ"] - qm["dHdQ"]) / (2 * step), ref["HQQ"][k], atol=1e-6)
        np.testing.assert_allclose((qp["dHdP"] - qm["dHdP"]) / (2 * step), ref["HQP"][k], atol=1e-6)
        np.testing.assert_allclose((pp["dHdP"] - pm["dHdP"]) / (2 * step), ref["HPP"][k], atol=1e-6)
        np.testing.assert_allclose((pp["dHdQ"] - pm["dHdQ"]) / (2 * step), ref["HPQ"][k], atol=1e-6)


# ---------------------------------------------------------------------------
# The interpolating prefilter (FGA_BSPLINE_INTERP)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [(False, False), (True, False), (True, True)])
def test_interp_coefficients_interpolate_the_samples(periodic):
    # the oracle's own spline evaluation (pinned above) at the grid points gives the samples
    n = (13, 11)
    g = O.Grid(n, (0.1, 0.2), (0.3, -0.4), periodic)
    rng = np.random.default_rng(21)
    c = 1.0 + rng.uniform(0.0, 1.0, n)
    C = O.interp_coefficients(g, c)
    axes = [g.o[k] + g.h[k] * np.arange(n[k]) for k in range(2)]
    X = np.stack([a.ravel() for a in np.meshgrid(*axes, indexing="ij")], axis=1)
    val, _, _, _ = O.medium_eval(g, C, X, order=0)
    np.testing.assert_allclose(val, c.ravel(), rtol=0, atol=1e-13)
    assert np.max(np.abs(C - c)) > 1e-3  # the prefilter does change the values


def test_interp_coefficients_periodic_equal_scipy_wrap_filter():
    from scipy import ndimage

    n = (16, 12)
    g = O.Grid(n, (1.0, 1.0), (0.0, 0.0), (True, True))
    c = np.random.default_rng(22).standard_normal(n)
    ref = ndimage.spline_filter(c, order=3, mode="grid-wrap")
    np.testing.assert_allclose(O.interp_coefficients(g, c), ref, atol=1e-12)
