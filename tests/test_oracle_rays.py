"""Pins of the oracle's ray, dynamic-ray, amplitude and action integration.

Facts used (none of them is the oracle's own formula):
  * homogeneous medium, any d: Q = q + sigma c t p/|p|, P = p,
    Z = 2I - i sigma (c t/|p|)(I - n n^T), a = sqrt(2) (2 - i sigma c t/|p|)^{(d-1)/2}
    (the exact solution of Eqs. characline, dzQ, dzP and a_formu for constant c);
  * variable medium: H = c(Q)|P| is constant along a ray; the quantity
    a^2/(c(Q)^2 det Z) is constant (the conservation statement after Eq. dzP), so
    a = c(Q)/c(q) sqrt(det Z) with a continuously chosen branch; the flow map is
    symplectic; A = d_z Q and B = d_z P agree with finite differences of whole
    rays in q and p (Eq. op_zZ); the action S stays zero (H is homogeneous of
    degree one in P); RK4 converges at fourth order;
  * the divided-difference form of Z (auxiliary rays offset by delta in q and p)
    is exact where the flow is affine and approaches the dynamic-ray Z at second
    order in delta.
"""

import cmath
import math

import numpy as np
import pytest

import oracle as O


def _open_grid(dim, n=40, h=0.25):
    return O.Grid((n,) * dim, (h,) * dim, (0.0,) * dim, (False,) * dim)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("sigma", [1, -1])
def test_homogeneous_closed_form(dim, sigma):
    c0 = 1.7
    g = _open_grid(dim)
    coef = np.full((40,) * dim, c0)
    rng = np.random.default_rng(10 + dim)
    nG = 12
    q = rng.uniform(4.0, 6.0, (nG, dim))
    p = rng.uniform(-1.5, 1.5, (nG, dim))
    p[0] = 0.05 * np.sign(p[0] + 1e-3)  # small |p|: fast amplitude change
    T, dt = 0.6, 1e-3
    nsteps = int(round(T / dt))
    st = O.propagate(g, coef, nsteps, dt, np.full(nG, sigma), q, p, nthreads=2)
    pn = np.linalg.norm(p, axis=1)
    nh = p / pn[:, None]
    t = nsteps * dt
    np.testing.assert_allclose(st["Q"], q + sigma * c0 * t * nh, atol=1e-12)
    np.testing.assert_allclose(st["P"], p, atol=1e-14)
    for i in range(nG):
        alpha = sigma * c0 * t / pn[i]
        proj = np.eye(dim) - np.outer(nh[i], nh[i])
        Aex = np.eye(dim) - 1j * alpha * proj
        np.testing.assert_allclose(st["A"][i], Aex, atol=1e-11)
        np.testing.assert_allclose(st["B"][i], -1j * np.eye(dim), atol=1e-14)
        aex = math.sqrt(2.0) * (2.0 - 1j * alpha) ** ((dim - 1) / 2.0)
        # RK4 truncation error grows with c dt/|p| (about 0.024 per step for ray 0)
        tol = 1e-9 if i == 0 else 1e-11
        assert abs(st["a"][i] - aex) <= tol * abs(aex), (i, st["a"][i], aex)
    assert np.max(np.abs(st["S"])) <= 1e-13


def _lens_medium(n=48, h=1.0 / 48):
    ax = h * np.arange(n)
    X, Z = np.meshgrid(ax, ax, indexing="ij")
    c = 1.0 + 0.3 * np.exp(-((X - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.02)
    return O.Grid((n, n), (h, h), (0.0, 0.0), (False, False)), c


def _rays_through_lens(g, c, nsteps, dt, sigma=1):
    # centres kept off the knot lines (the spline's third derivative jumps there)
    q = np.array([[0.351, 0.203], [0.507, 0.253], [0.622, 0.301], [0.451, 0.803], [0.303, 0.507]])
    p = np.array([[0.1, 1.0], [0.0, 0.7], [-0.2, 0.9], [0.3, -1.1], [1.2, 0.05]])
    st = O.propagate(g, c, nsteps, dt, np.full(len(q), sigma), q, p, nthreads=2)
    return q, p, st


@pytest.mark.parametrize("sigma", [1, -1])
def test_variable_medium_invariants(sigma):
    g, c = _lens_medium()
    dt = 5e-4
    # integrate in segments so that the branch of sqrt(det Z) can be followed
    q, p, _ = _rays_through_lens(g, c, 0, dt, sigma)
    cq, _, _, _ = O.medium_eval(g, c, q, order=0)
    H0 = cq * np.linalg.norm(p, axis=1)
    prev_arg = np.zeros(len(q))
    arg_acc = np.zeros(len(q))
    for seg in range(1, 9):
        nsteps = 100 * seg
        _, _, st = _rays_through_lens(g, c, nsteps, dt, sigma)
        cQ, _, _, _ = O.medium_eval(g, c, st["Q"], order=0)
        H = cQ * np.linalg.norm(st["P"], axis=1)
        np.testing.assert_allclose(H, H0, rtol=1e-9)
        Z = st["A"] + 1j * st["B"]
        detZ = np.linalg.det(Z)
        inv = st["a"] ** 2 / (cQ ** 2 * detZ)
        np.testing.assert_allclose(inv, 1.0 / cq ** 2, rtol=1e-9)
        # continuous arg of det Z -> branch of the square root
        ang = np.angle(detZ)
        dang = np.angle(np.exp(1j * (ang - prev_arg)))
        arg_acc += dang
        prev_arg = ang
        a_closed = cQ / cq * np.sqrt(np.abs(detZ)) * np.exp(0.5j * arg_acc)
        np.testing.assert_allclose(st["a"], a_closed, rtol=1e-9)
        assert np.max(np.abs(st["S"])) < 1e-13


def test_variable_medium_symplectic_and_fd_jacobian():
    g, c = _lens_medium()
    dt, nsteps = 1e-3, 300
    q, p, st = _rays_through_lens(g, c, nsteps, dt)
    d = 2
    # (A)_{jk} = d_{z_j} Q_k = dQ_k/dq_j - i dQ_k/dp_j ;  (B)_{jk} = dP_k/dq_j - i dP_k/dp_j
    dQdq = st["A"].real.transpose(0, 2, 1)
    dQdp = -st["A"].imag.transpose(0, 2, 1)
    dPdq = st["B"].real.transpose(0, 2, 1)
    dPdp = -st["B"].imag.transpose(0, 2, 1)
    h = 1e-6
    for j in range(d):
        e = np.zeros(d)
        e[j] = h
        stp = O.propagate(g, c, nsteps, dt, np.ones(len(q)), q + e, p, nthreads=2)
        stm = O.propagate(g, c, nsteps, dt, np.ones(len(q)), q - e, p, nthreads=2)
        np.testing.assert_allclose((stp["Q"] - stm["Q"]) / (2 * h), dQdq[:, :, j], atol=2e-7)
        np.testing.assert_allclose((stp["P"] - stm["P"]) / (2 * h), dPdq[:, :, j], atol=2e-7)
        stp = O.propagate(g, c, nsteps, dt, np.ones(len(q)), q, p + e, nthreads=2)
        stm = O.propagate(g, c, nsteps, dt, np.ones(len(q)), q, p - e, nthreads=2)
        np.testing.assert_allclose((stp["Q"] - stm["Q"]) / (2 * h), dQdp[:, :, j], atol=2e-7)
        np.testing.assert_allclose((stp["P"] - stm["P"]) / (2 * h), dPdp[:, :, j], atol=2e-7)
    J = np.block([[dQdq, dQdp], [dPdq, dPdp]])
    Om = np.block([[np.zeros((d, d)), np.eye(d)], [-np.eye(d), np.zeros((d, d))]])
    for i in range(len(q)):
        np.testing.assert_allclose(J[i].T @ Om @ J[i], Om, atol=1e-10)


def test_rk4_fourth_order():
    # A linear velocity is reproduced exactly by the spline, so the right-hand side is
    # smooth and RK4 must show its fourth order (across the knots of a general spline
    # the Hessian of c only has kinks, which lowers the observed order).
    n, h = 64, 1.0 / 16
    ax = h * np.arange(n)
    X, Z = np.meshgrid(ax, ax, indexing="ij")
    c = 1.0 + 0.5 * X - 0.2 * Z
    g = O.Grid((n, n), (h, h), (0.0, 0.0), (False, False))
    q = np.array([[1.3, 2.0], [2.2, 1.7], [1.9, 2.4]])
    p = np.array([[0.2, 1.0], [-0.6, 0.3], [0.05, -0.9]])
    T = 1.0
    ref = O.propagate(g, c, 3200, T / 3200, np.ones(3), q, p, nthreads=1)
    errs = []
    for nst in (40, 80):
        st = O.propagate(g, c, nst, T / nst, np.ones(3), q, p, nthreads=1)
        errs.append(np.max(np.abs(st["Q"] - ref["Q"])) + np.max(np.abs(st["a"] - ref["a"])))
    ratio = errs[0] / errs[1]
    assert 12.0 < ratio < 20.0, (errs, ratio)


def test_periodic_wrap_of_centres():
    n, h = 32, 1.0 / 32
    g = O.Grid((n, n), (h, h), (0.0, 0.0), (True, True))
    coef = np.ones((n, n))
    q = np.array([[0.9, 0.05]])
    p = np.array([[1.0, -1.0]])
    st = O.propagate(g, coef, 200, 1e-3, np.array([1]), q, p, nthreads=1)
    exp = np.mod(q + 0.2 * p / np.linalg.norm(p), 1.0)
    np.testing.assert_allclose(st["Q"], exp, atol=1e-13)


# ---------------------------------------------------------------------------
# The divided-difference alternative for d_z Q, d_z P (the passage after Eq. op_zZ)
# ---------------------------------------------------------------------------

def test_divided_differences_homogeneous_closed_form():
    # constant c: Q = q + c t p/|p| is linear in q, and in p up to the curvature of p/|p|,
    # so the central differences are exact in q (and in 1D) and carry an O(delta^2) error
    # in p: the amplitude error must fall by 4 when delta halves, against the closed form
    for dim in (1, 2, 3):
        g = _open_grid(dim)
        c0 = 1.7
        coef = np.full((40,) * dim, c0)
        rng = np.random.default_rng(3)
        q = rng.uniform(4.0, 6.0, (6, dim))
        p = rng.uniform(-1.5, 1.5, (6, dim))
        T, dt = 0.6, 1e-3
        sig = np.ones(6, np.int32)
        pn = np.linalg.norm(p, axis=1)
        aex = math.sqrt(2.0) * (2.0 - 1j * c0 * T / pn) ** ((dim - 1) / 2.0)
        dyn = O.propagate(g, coef, 600, dt, sig, q, p, nthreads=2)
        errs = []
        for delta in (1e-2, 5e-3, 2.5e-3):
            st = O.propagate_dd(g, coef, 600, dt, sig, q, p, delta, delta, nthreads=2)
            assert np.array_equal(st["Q"], dyn["Q"]) and np.array_equal(st["P"], dyn["P"])
            np.testing.assert_allclose(st["B"], np.broadcast_to(-1j * np.eye(dim), st["B"].shape),
                                       atol=1e-13)
            errs.append(np.max(np.abs(st["a"] - aex)))
        if dim == 1:
            assert max(errs) <= 1e-14
        else:
            assert errs[0] <= 1.1e-3
            for e0, e1 in zip(errs, errs[1:]):
                assert 3.9 <= e0 / e1 <= 4.1, errs


def test_divided_differences_converge_to_dynamic_rays():
    # variable medium: Z from differences of the discrete flow tends to the dynamic-ray Z
    # (the Jacobian of the same RK4 flow) at second order in delta; the spline's third
    # derivative jumps at knots, so the observed ratio per halving sits a little under 4
    g, c = _lens_medium(64, 1.0 / 64)
    q = np.array([[0.351, 0.203], [0.507, 0.253], [0.622, 0.301], [0.451, 0.803]])
    p = np.array([[0.1, 1.0], [0.0, 0.7], [-0.2, 0.9], [0.3, -1.1]])
    sig = np.ones(4, np.int32)
    dyn = O.propagate(g, c, 400, 1e-3, sig, q, p, nthreads=2)
    diffs = []
    for delta in (2e-3, 1e-3, 5e-4):
        st = O.propagate_dd(g, c, 400, 1e-3, sig, q, p, delta, delta, nthreads=2)
        diffs.append(np.max(np.abs(st["a"] - dyn["a"])))
        np.testing.assert_allclose(st["A"], dyn["A"], atol=100 * delta ** 2)
    assert diffs[-1] <= 1e-4
    for e0, e1 in zip(diffs, diffs[1:]):
        assert 2.8 <= e0 / e1 <= 4.2, diffs
