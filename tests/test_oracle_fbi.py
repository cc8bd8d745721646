"""Pins of the oracle's FBI transform (Initial wavefield decomposition section).

* The FFT-on-the-box route (the paper's fast FBI) agrees with the brute-force
  direct sum of the definition, written with the phase exponent itself.
* For Gaussian data the transform has a closed form (a Gaussian integral), which
  pins the h^d factor, the sign of the phase, the p values and the window.
"""

import math

import numpy as np
import pytest

import oracle as O


def _rand_data(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)


@pytest.mark.parametrize("case", [
    dict(n=(40,), h=(0.05,), per=(False,), eps=0.01, s=(3,), box=(16,)),
    dict(n=(24,), h=(1.0 / 24,), per=(True,), eps=0.004, s=(4,), box=(24,)),
    dict(n=(18, 14), h=(0.1, 0.08), per=(False, False), eps=0.02, s=(4, 3), box=(8, 10)),
    dict(n=(16, 12), h=(1.0 / 16, 0.1), per=(True, False), eps=0.01, s=(4, 3), box=(16, 8)),
    dict(n=(9, 8, 7), h=(0.1, 0.125, 0.11), per=(False, True, False), eps=0.02, s=(3, 2, 3),
         box=(6, 8, 4)),
])
def test_fft_route_matches_direct_sum(case):
    g = O.Grid(case["n"], case["h"], (0.0,) * len(case["n"]), case["per"])
    f = _rand_data(case["n"], 7)
    psi = O.fbi(g, f, case["eps"], case["s"], case["box"])
    nq = O.q_counts(g, case["s"])
    qi_multi = np.stack(np.unravel_index(np.arange(int(np.prod(nq))), tuple(nq)), axis=1)
    qi = qi_multi * np.array(case["s"])[None, :]
    pp = O.p_points(g, case["eps"], case["box"])
    # every (q, p) pair
    QI = np.repeat(qi, pp.shape[0], axis=0)
    PV = np.tile(pp, (qi.shape[0], 1))
    direct = O.fbi_direct(g, f, case["eps"], case["box"], QI, PV).reshape(psi.shape)
    scale = np.max(np.abs(direct))
    assert np.max(np.abs(psi - direct)) <= 1e-13 * scale


def test_gaussian_data_closed_form_2d():
    # f(y) = exp(-|y - y0|^2/(2 s^2)); per axis the transform is the Gaussian integral
    #   int exp(-(y-y0)^2/(2 s^2) - (y-q)^2/(2 eps) - i p (y-q)/eps) dy
    #     = sqrt(2 pi/alpha) exp(beta^2/(2 alpha) - y0^2/(2 s^2) - q^2/(2 eps) + i p q/eps),
    #   alpha = 1/s^2 + 1/eps,  beta = y0/s^2 + (q - i p)/eps.
    n = (96, 80)
    h = (0.01, 0.0125)
    g = O.Grid(n, h, (0.0, 0.0), (False, False))
    eps = 0.004
    sg = 0.05  # resolved: its spectrum at the grid Nyquist is below e^{-70}
    y0 = (0.47, 0.51)
    xs = [h[k] * np.arange(n[k]) for k in range(2)]
    X, Z = np.meshgrid(*xs, indexing="ij")
    f = np.exp(-((X - y0[0]) ** 2 + (Z - y0[1]) ** 2) / (2 * sg ** 2))
    s = (4, 4)
    box = (96, 80)
    psi = O.fbi(g, f, eps, s, box)
    qp = O.q_points(g, s)
    pp = O.p_points(g, eps, box)
    # only q near the data, so that the box truncation (e^{-(L/2)^2/(2 eps)}) is negligible
    near = np.where(np.max(np.abs(qp - np.array(y0)[None, :]), axis=1) < 0.08)[0]
    assert near.size > 10
    ex = np.ones((near.size, pp.shape[0]), dtype=complex)
    for k in range(2):
        q = qp[near, k][:, None]
        p = pp[:, k][None, :]
        alpha = 1.0 / sg ** 2 + 1.0 / eps
        beta = y0[k] / sg ** 2 + (q - 1j * p) / eps
        ex *= (math.sqrt(2 * math.pi / alpha)
               * np.exp(beta ** 2 / (2 * alpha) - y0[k] ** 2 / (2 * sg ** 2) - q ** 2 / (2 * eps)
                        + 1j * p * q / eps))
    got = psi[near]
    assert np.max(np.abs(got - ex)) <= 1e-12 * np.max(np.abs(ex))


def test_gaussian_data_closed_form_3d():
    # the 3D transform of a Gaussian is the product of three 1D Gaussian integrals
    # (the closed form of the 2D test per axis); only q near the data (q_subset). The
    # data sit 8 sg from the grid's edges, the box (+-8 sqrt(eps)) cuts the window at
    # e^{-32}, and the integrand's spectrum at the grid Nyquist is below e^{-24}.
    n = (80, 76, 72)
    h = (0.0125, 0.0125, 0.0125)
    g = O.Grid(n, h, (0.0, 0.0, 0.0), (False, False, False))
    eps = 0.001
    sg = 0.06
    y0 = (0.5, 0.47, 0.45)
    xs = [h[k] * np.arange(n[k]) for k in range(3)]
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    f = np.exp(-((X - y0[0]) ** 2 + (Y - y0[1]) ** 2 + (Z - y0[2]) ** 2) / (2 * sg ** 2))
    s = (4, 4, 4)
    box = (40, 40, 40)
    qp_all = O.q_points(g, s)
    near = np.where(np.max(np.abs(qp_all - np.array(y0)[None, :]), axis=1) < 0.05)[0]
    assert near.size >= 8
    psi = O.fbi(g, f, eps, s, box, q_subset=near)
    pp = O.p_points(g, eps, box)
    ex = np.ones((near.size, pp.shape[0]), dtype=complex)
    for k in range(3):
        q = qp_all[near, k][:, None]
        p = pp[:, k][None, :]
        alpha = 1.0 / sg ** 2 + 1.0 / eps
        beta = y0[k] / sg ** 2 + (q - 1j * p) / eps
        ex *= (math.sqrt(2 * math.pi / alpha)
               * np.exp(beta ** 2 / (2 * alpha) - y0[k] ** 2 / (2 * sg ** 2) - q ** 2 / (2 * eps)
                        + 1j * p * q / eps))
    assert np.max(np.abs(psi - ex)) <= 1e-10 * np.max(np.abs(ex))


def test_p_grid_is_symmetric_and_excludes_zero():
    g = O.Grid((20, 16), (0.1, 0.1), (0, 0), (False, False))
    box = (8, 6)
    v = O.p_valid(box)
    pp = O.p_points(g, 0.02, box)
    assert v.sum() == 7 * 5 - 1
    assert not np.any(np.all(pp[v] == 0, axis=1))
    key = {tuple(np.round(p, 12)) for p in pp[v]}
    assert all(tuple(np.round(-np.array(p), 12)) in key for p in key)
