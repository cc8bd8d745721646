"""Pin of the finite-difference reference used by the accuracy-versus-N sweep.

Constant speed c, radially symmetric Gaussian data u0 = exp(-r^2/(2 s^2)), u1 = 0: the
exact 2D solution is the Hankel transform
    u(r, t) = s^2 int_0^inf exp(-s^2 k^2/2) cos(c k t) J0(k r) k dk
(u^(k) = u0^(k) cos(c|k|t) with u0^(k) = 2 pi s^2 exp(-s^2|k|^2/2)), evaluated here by
the trapezoidal rule on a k grid reaching exp(-98). A wrong weight, a dropped c^2 or a
wrong time step changes the field by far more than the tolerance.
"""

import numpy as np
import pytest
from scipy.special import j0

import fd_reference as FD


def _hankel_exact(r, c0, s, t):
    k = np.linspace(0.0, 14.0 / s, 6001)
    w = np.full(k.size, k[1] - k[0])
    w[0] *= 0.5
    w[-1] *= 0.5
    ru, inv = np.unique(np.round(r, 12), return_inverse=True)
    g = np.exp(-0.5 * (s * k) ** 2) * np.cos(c0 * k * t) * k * w
    return (s * s * (j0(np.outer(ru, k)) @ g))[inv]


@pytest.mark.parametrize("refine", [2, 3])
def test_constant_speed_gaussian_matches_hankel_solution(refine):
    n, h, c0, s, xc, T = (121, 121), (0.01, 0.01), 2.0, 0.04, (0.6, 0.6), 0.15
    u, info = FD.solve(np.full(n, c0), h, n,
                       lambda X, Z: np.exp(-((X - xc[0]) ** 2 + (Z - xc[1]) ** 2) / (2 * s * s)),
                       lambda X, Z: np.zeros_like(X), T, refine=refine, pad=0.2)
    X, Z = np.meshgrid(np.arange(n[0]) * h[0], np.arange(n[1]) * h[1], indexing="ij")
    uex = _hankel_exact(np.hypot(X - xc[0], Z - xc[1]).ravel(), c0, s, T).reshape(n)
    assert np.linalg.norm(u - uex) <= 1e-4 * np.linalg.norm(uex)


def test_spline_velocity_is_the_clamped_bspline():
    # values at the knots of a linear ramp are the ramp (the B-spline reproduces linear
    # data), and beyond the grid the clamped coefficients give the edge value
    n = (10, 8)
    h = (0.5, 0.5)
    coef = np.add.outer(np.arange(n[0]) * 1.0, np.zeros(n[1])) + 3.0
    x = np.array([1.0, 2.25, 3.5, -5.0, 20.0])
    z = np.array([1.0, 1.5, 2.0, 1.0, 1.0])
    c = FD.spline_velocity(coef, h, x, z)
    assert np.allclose(c[:3], 3.0 + x[:3] / h[0], atol=1e-13)
    assert abs(c[3] - 3.0) <= 1e-13 and abs(c[4] - (3.0 + n[0] - 1)) <= 1e-13
