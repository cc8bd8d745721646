"""Pins of the oracle's forward-mode (tangent-linear) derivative along a change V of
the velocity coefficients, the Gaussian set held fixed.

The derivative is the dual-number evaluation of the oracle's own RK4 (Eqs.
characline, dzQ, dzP, a_formu, the action) and reconstruction sum (Eq. recons),
plus the derivative of the branch split of Eq. psi through c(q), written out. It is
pinned against what does not come from it:
* its value part is the plain oracle, bit for bit;
* for constant speed the rays, the dynamic rays and the amplitude have closed forms
  (Q = q + sigma c t p/|p|, A = I - i sigma c t/|p| (I - n n^T), B = -iI,
  a = sqrt(2) (2 - i sigma c t/|p|)^{(d-1)/2}), and so does their derivative in c;
  the traces' derivative then follows term by term, including the branch split;
* in a variable medium it equals Richardson-extrapolated central differences of the
  plain oracle (rays, dynamic rays, amplitude, traces).
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import workloads as WL


def _lens(T=0.06, dt=2e-3, tau=2e-2):
    # the lens of the adjoint tests, centre off the spline's knot lines
    return WL.lens_2d(N=48, eps=1.0 / 300, T=T, dt=dt, s=2, box=32, tau=tau, kappa=8.0,
                      k0=20 * math.pi, width2=0.006, x0=(0.4937, 0.33), center=(0.5071, 0.4963))


def _grid(pr):
    return O.Grid(pr.n, pr.h, pr.origin, pr.periodic)


def _direction(n, seed):
    rng = np.random.default_rng(seed)
    axes = np.meshgrid(*[np.linspace(0, 1, m) for m in n], indexing="ij")
    v = np.zeros(n)
    for _ in range(4):
        ph = sum(rng.uniform(1, 4) * a for a in axes) + rng.uniform()
        v += rng.standard_normal() * np.sin(2 * np.pi * ph)
    return v / np.abs(v).max()


def _richardson(f, h):
    """Fourth-order central difference (8 (f(h) - f(-h)) - (f(2h) - f(-2h)))/(12 h)."""
    return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)


def _rays(pr, n=24, seed=0):
    sh = pr.shots[0]
    g = _grid(pr)
    dec = O.decompose(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, pr.tau)
    gs = dec["gauss"]
    pick = np.random.default_rng(seed).choice(gs["sigma"].size, n, replace=False)
    return g, dec, gs["sigma"][pick], gs["q"][pick], gs["p"][pick]


def test_value_part_is_the_plain_oracle_bitwise():
    pr = _lens()
    g, dec, sg, q, p = _rays(pr)
    V = _direction(pr.n, 1)
    st, _ = O.propagate_tangent(g, pr.velocity, V, pr.nsteps, pr.dt, sg, q, p)
    ref = O.propagate(g, pr.velocity, pr.nsteps, pr.dt, sg, q, p)
    for k in ref:
        assert np.array_equal(st[k], ref[k]), k
    sh = pr.shots[0]
    gs = dec["gauss"]
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    xr = np.stack([np.linspace(0.2, 0.8, 7), np.full(7, 0.45)], axis=1)
    tr, _ = O.traces_tangent(g, pr.velocity, V, pr.nsteps, pr.dt, 5, gs["sigma"], gs["q"],
                             gs["p"], gs["psi"], np.zeros_like(gs["psi"]), sh.eps, pr.kappa, W, xr)
    ref_tr = O.traces(g, pr.velocity, pr.nsteps, pr.dt, 5, gs["sigma"], gs["q"], gs["p"],
                      gs["psi"], sh.eps, pr.kappa, W, xr)
    assert np.array_equal(tr, ref_tr)


@pytest.mark.parametrize("dim", [2, 3])
def test_propagate_tangent_constant_speed_closed_form(dim):
    # c = c0 everywhere (constant coefficients: the clamped spline is c0 on all of R^d)
    # and V = 1: the derivative in c0 of the closed-form rays and amplitude
    n = (20,) * dim
    h = (0.05,) * dim
    g = O.Grid(n, h, (0.0,) * dim, (False,) * dim)
    c0 = 1.3
    C = np.full(n, c0)
    V = np.ones(n)
    rng = np.random.default_rng(dim)
    m = 12
    q = rng.uniform(0.3, 0.7, (m, dim))
    p = rng.standard_normal((m, dim))
    p *= (rng.uniform(0.7, 1.5, m) / np.linalg.norm(p, axis=1))[:, None]  # |p| away from 0
    sg = np.where(rng.uniform(size=m) < 0.5, 1, -1).astype(np.int32)
    nsteps, dt = 40, 5e-3
    t = nsteps * dt
    st, dst = O.propagate_tangent(g, C, V, nsteps, dt, sg, q, p)
    pn = np.linalg.norm(p, axis=1)
    nh = p / pn[:, None]
    s = sg.astype(float)
    proj = np.eye(dim)[None] - nh[:, :, None] * nh[:, None, :]
    # values
    assert np.max(np.abs(st["Q"] - (q + (s * c0 * t)[:, None] * nh))) <= 1e-13
    assert np.max(np.abs(st["A"] - (np.eye(dim)[None] - (1j * s * c0 * t / pn)[:, None, None]
                                    * proj))) <= 1e-13
    w = 2.0 - 1j * s * c0 * t / pn
    a = math.sqrt(2.0) * w ** ((dim - 1) / 2.0)
    assert np.max(np.abs(st["a"] - a) / np.abs(a)) <= 1e-10
    # derivatives in c0
    assert np.max(np.abs(dst["Q"] - (s * t)[:, None] * nh)) <= 1e-13
    assert np.max(np.abs(dst["P"])) <= 1e-13
    assert np.max(np.abs(dst["A"] + (1j * s * t / pn)[:, None, None] * proj)) <= 1e-13
    assert np.max(np.abs(dst["B"])) <= 1e-13
    da = a * (dim - 1) / 2.0 * (-1j * s * t / pn) / w
    assert np.max(np.abs(dst["a"] - da)) <= 1e-10 * np.max(np.abs(da))
    assert np.max(np.abs(dst["S"])) <= 1e-13


def test_propagate_tangent_matches_richardson_differences():
    pr = _lens()
    g, dec, sg, q, p = _rays(pr, n=24, seed=3)
    for seed in (1, 2):
        V = _direction(pr.n, seed)
        st, dst = O.propagate_tangent(g, pr.velocity, V, pr.nsteps, pr.dt, sg, q, p)
        for key in ("Q", "P", "A", "B", "a"):
            fd = _richardson(lambda e: O.propagate(g, pr.velocity + e * V, pr.nsteps, pr.dt, sg,
                                                   q, p)[key], 1e-4)
            scale = np.max(np.abs(dst[key]))
            assert scale > 0, key
            # steps of 1e-4: larger ones move rays across the spline's knot lines, where
            # the Hessian of c has kinks and the differences lose their order
            assert np.max(np.abs(dst[key] - fd)) <= 1e-9 * scale, key


def test_traces_tangent_matches_richardson_differences():
    pr = _lens()
    sh = pr.shots[0]
    g, dec, _, _, _ = _rays(pr)
    gs = dec["gauss"]
    keys = (gs["sigma"], gs["qidx"], gs["pidx"])
    xr = np.stack([np.linspace(0.2, 0.8, 9), np.full(9, 0.42)], axis=1)
    for seed in (4, 5):
        V = _direction(pr.n, seed)
        tr, dtr = O.frozen_set_traces_tangent(g, pr.velocity, V, sh.u0, sh.u1, sh.eps, sh.q_stride,
                                              sh.box, keys, pr.nsteps, pr.dt, 5, pr.kappa, xr)
        ref = O.frozen_set_traces(g, pr.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, keys,
                                  pr.nsteps, pr.dt, 5, pr.kappa, xr)
        assert np.array_equal(tr, ref)
        fd = _richardson(lambda e: O.frozen_set_traces(g, pr.velocity + e * V, sh.u0, sh.u1, sh.eps,
                                                       sh.q_stride, sh.box, keys, pr.nsteps, pr.dt,
                                                       5, pr.kappa, xr), 2e-4)
        err = np.linalg.norm(dtr.real - fd.real) / np.linalg.norm(fd.real)
        assert err <= 1e-7, err
        # the derivative of real data's field stays real (both branches summed)
        assert np.linalg.norm(dtr.imag) <= 1e-10 * np.linalg.norm(dtr.real)


def test_branch_split_tangent_against_differences():
    pr = _lens()
    sh = pr.shots[0]
    g = _grid(pr)
    rows = np.arange(40, 60)
    psi0 = O.fbi(g, sh.u0, sh.eps, sh.q_stride, sh.box, q_subset=rows)
    psi1 = O.fbi(g, sh.u1, sh.eps, sh.q_stride, sh.box, q_subset=rows)
    V = _direction(pr.n, 6)
    dp, dm = O.branch_split_tangent(g, pr.velocity, V, sh.eps, sh.q_stride, sh.box, psi1, rows)
    fp = _richardson(lambda e: O.branch_split(g, pr.velocity + e * V, sh.eps, sh.q_stride, sh.box,
                                              psi0, psi1, rows)[0], 1e-3)
    fm = _richardson(lambda e: O.branch_split(g, pr.velocity + e * V, sh.eps, sh.q_stride, sh.box,
                                              psi0, psi1, rows)[1], 1e-3)
    assert np.max(np.abs(dp - fp)) <= 1e-10 * np.max(np.abs(dp))
    assert np.max(np.abs(dm - fm)) <= 1e-10 * np.max(np.abs(dm))
    assert np.max(np.abs(dp + dm)) <= 1e-15 * np.max(np.abs(dp))  # psi0 does not move


def test_traces_tangent_constant_speed_closed_form():
    # open 2D grid, c = c0, V = 1; every kept Gaussian's term and its c0-derivative in
    # closed form (rays, amplitude, branch split), summed at the receivers
    N = 40
    h = 1.0 / N
    g = O.Grid((N, N), (h, h), (0.0, 0.0), (False, False))
    c0 = 1.2
    C = np.full((N, N), c0)
    V = np.ones((N, N))
    ax = h * np.arange(N)
    X, Z = np.meshgrid(ax, ax, indexing="ij")
    env = np.exp(-((X - 0.5) ** 2 + (Z - 0.4) ** 2) / 0.008)
    u0 = env * np.cos(16 * math.pi * Z)
    u1 = env * np.sin(16 * math.pi * Z) * 3.0
    eps, s, box, tau, kappa = 1.0 / 300, (2, 2), (32, 32), 2e-2, 7.0
    dec = O.decompose(g, C, u0, u1, eps, s, box, tau)
    gs = dec["gauss"]
    nsteps, dt, rec = 30, 2e-3, 10
    xr = np.stack([np.linspace(0.3, 0.7, 6), np.full(6, 0.45)], axis=1)
    W = O.quadrature_weight(g, eps, s, box)
    keys = (gs["sigma"], gs["qidx"], gs["pidx"])
    tr, dtr = O.frozen_set_traces_tangent(g, C, V, u0, u1, eps, s, box, keys, nsteps, dt, rec,
                                          kappa, xr)
    sg = gs["sigma"].astype(float)
    q, p, psi = gs["q"], gs["p"], gs["psi"]
    psi1 = dec["psi1"][gs["qidx"], gs["pidx"]]
    pn = np.linalg.norm(p, axis=1)
    nh = p / pn[:, None]
    dpsi = -sg * 0.5j * eps * psi1 / (c0 * c0 * pn)
    norm = (2 * math.pi * eps) ** (-3.0)
    cut = kappa * math.sqrt(eps)
    ref = np.zeros(dtr.shape, dtype=complex)
    dref = np.zeros(dtr.shape, dtype=complex)
    for m in range(nsteps // rec + 1):
        t = m * rec * dt
        Q = q + (sg * c0 * t)[:, None] * nh
        dQ = (sg * t)[:, None] * nh
        w = 2.0 - 1j * sg * c0 * t / pn
        a = math.sqrt(2.0) * np.sqrt(w)
        da = a * 0.5 * (-1j * sg * t / pn) / w
        for r in range(xr.shape[0]):
            dx = xr[r][None, :] - Q
            inside = np.all(np.abs(dx) <= cut, axis=1)
            E = 1j * np.sum(p * dx, axis=1) / eps - np.sum(dx * dx, axis=1) / (2 * eps)
            dE = np.sum((-1j * p + dx) * dQ, axis=1) / eps
            term = W * norm * np.exp(E)
            ref[m, r] = np.sum(np.where(inside, term * a * psi, 0.0))
            dref[m, r] = np.sum(np.where(inside, term * (dpsi * a + psi * da + psi * a * dE), 0.0))
    assert np.linalg.norm(tr - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(dtr - dref) <= 1e-9 * np.linalg.norm(dref)
