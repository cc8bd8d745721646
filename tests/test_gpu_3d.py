"""The 3D path (d = 3, FP64) against the FP64 CPU oracle, element by element: the
three-stage FBI with the branch split, the Gaussian set, the 45-value ray states and the
field on a 20^3 grid (two 16-point tiles per axis, the second ragged); the traces recorded
inside the 3D ray kernel at receiver points against the oracle's traces; the 3D adjoint
against the oracle's forward-mode derivative (dot-product test)."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL
from test_gpu_parity import FIELD_TOL, _grid, check_decomposition, check_rays, oracle_field, rel, run_gpu

pytestmark = pytest.mark.gpu


def _problem(**kw):
    args = dict(N=20, eps=0.0025, s=2, box=12, tau=5e-2, T=0.02, k0=4 * math.pi, width2=0.01)
    args.update(kw)
    return WL.lens_3d(**args)


def test_lens_3d_elementwise():
    prob = _problem()
    plan, counts, u = run_gpu(prob)
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    qi, pi = check_decomposition(plan, prob, dec)
    assert counts[0] == int(np.sum(dec["gauss"]["sigma"] == 1)) and counts[0] > 1000
    check_rays(plan, prob, 0, qi[::53], pi[::53], tol_q=1e-12, tol_a=1e-11)
    uo = oracle_field(prob, 0, dec, prob.grid_points())
    assert np.linalg.norm(uo.imag) <= 1e-12 * np.linalg.norm(uo.real)
    assert rel(u[0].ravel(), uo.real) <= FIELD_TOL
    assert np.abs(u[0].ravel() - uo.real).max() <= FIELD_TOL * np.abs(uo.real).max()
    plan.close()


def test_lens_3d_box_above_64_points():
    """Boxes of 72 points per axis on a 32^3 lens (q-stride 8: 4^3 q, 373 248 p per q):
    psi+ element by element against the oracle's FFT route, the kept set outside the guard
    band, sampled rays, and the field at 4000 sampled grid points against the oracle's
    sum over every kept Gaussian of both branches."""
    prob = WL.lens_3d(N=32, eps=0.012, s=8, box=72, tau=5e-2, T=0.01, k0=10 * math.pi,
                      width2=0.02)
    plan, counts, u = run_gpu(prob)
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    qi, pi = check_decomposition(plan, prob, dec)
    assert counts[0] > 10000
    check_rays(plan, prob, 0, qi[::97], pi[::97], tol_q=1e-12, tol_a=1e-11)
    rng = np.random.default_rng(5)
    pts = prob.grid_points()
    pick = rng.choice(pts.shape[0], 4000, replace=False)
    uo = oracle_field(prob, 0, dec, pts[pick])
    assert np.linalg.norm(uo.imag) <= 1e-12 * np.linalg.norm(uo.real)
    assert rel(u[0].ravel()[pick], uo.real) <= FIELD_TOL
    plan.close()


def test_lens_3d_hamiltonian_conserved():
    """T = 0.1 s (100 RK4 steps): c(Q)|P| (the Hamiltonian of the + branch) stays within
    1e-8 of its initial value along every ray, and every state is finite."""
    prob = _problem(T=0.1)
    plan, counts, u = run_gpu(prob)
    st = plan.state(0)
    qi, pi, _ = plan.gaussians(0)
    sh = prob.shots[0]
    g = _grid(prob)
    q = O.q_points(g, sh.q_stride)[qi]
    p = O.p_points(g, sh.eps, sh.box)[pi]
    c0, _, _, _ = O.medium_eval(g, prob.velocity, q, order=0)
    c1, _, _, _ = O.medium_eval(g, prob.velocity, st["Q"], order=0)
    H0 = c0 * np.linalg.norm(p, axis=1)
    H1 = c1 * np.linalg.norm(st["P"], axis=1)
    assert np.max(np.abs(H1 - H0) / H0) <= 1e-8
    assert np.all(np.isfinite(u)) and np.all(np.isfinite(st["A"])) and np.all(np.isfinite(st["a"]))
    plan.close()


REC = 5


def _receivers_3d():
    """Two 5 x 5 layers of receivers across the packet's path (z = 0.35, 0.42) and a few
    loose points, spread over both 16-point tiles of each axis."""
    g = np.linspace(0.38, 0.62, 5)
    X, Y = np.meshgrid(g, g, indexing="ij")
    layers = [np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1) for z in (0.35, 0.42)]
    loose = np.array([[0.5, 0.5, 0.5], [0.81, 0.47, 0.37], [0.2, 0.9, 0.4], [0.55, 0.52, 0.95]])
    return np.ascontiguousarray(np.concatenate(layers + [loose]))


def test_traces_3d_match_oracle():
    """Re u at 54 receivers every 5 steps to T = 0.02 s, recorded by the 3D ray kernel,
    against the oracle's traces of the same Gaussians (both branches summed literally by
    the oracle): rel-L2 <= 1e-10."""
    import torch

    prob = _problem()
    xr = _receivers_3d()
    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True)
    plan.set_receivers(xr, REC)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    tr = plan.traces()
    plan.close()
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    gs = dec["gauss"]
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    ot = O.traces(g, prob.velocity, prob.nsteps, prob.dt, REC, gs["sigma"], gs["q"], gs["p"],
                  gs["psi"], sh.eps, prob.kappa, W, xr)
    assert np.linalg.norm(ot.imag) <= 1e-12 * np.linalg.norm(ot.real)
    assert np.linalg.norm(ot.real) > 0
    err = np.linalg.norm(tr[0] - ot.real) / np.linalg.norm(ot.real)
    print("3D traces vs oracle: rel-L2 %.3e" % err)
    assert err <= 1e-10, err


def _smooth_direction_3d(n, seed):
    rng = np.random.default_rng(seed)
    ax = [np.linspace(0, 1, k) for k in n]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    v = np.zeros(n)
    for _ in range(4):
        kx, ky, kz = rng.uniform(1, 3, 3)
        v += rng.standard_normal() * (np.sin(2 * np.pi * (kx * X + rng.uniform())) *
                                      np.cos(2 * np.pi * (ky * Y + rng.uniform())) *
                                      np.sin(2 * np.pi * (kz * Z + rng.uniform())))
    return v / np.abs(v).max()


def test_adjoint_3d_against_oracle_tangent():
    """The 3D adjoint (reverse mode through the 45-value ray state, the 64-tap spline with
    its third derivatives and the 3 x 3 cofactor form of tr(Z^-1 dZ/dt)) against the
    oracle's forward mode on the same frozen set: <fga_grad(w), v> = <w, Re J v> for
    w = the traces and a random w, along a smooth v and the two cells where the gradient
    is largest, <= 1e-12 relative."""
    import torch

    prob = _problem()
    xr = _receivers_3d()
    c = prob.velocity
    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True)
    plan.set_receivers(xr, REC)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    tr = plan.traces()
    qi, pi, _ = plan.gaussians(0)
    keys = set(zip(qi.tolist(), pi.tolist()))
    rng = np.random.default_rng(11)
    ws = [np.ascontiguousarray(tr), rng.standard_normal(tr.shape)]
    grads = [plan.grad(np.ascontiguousarray(w)) for w in ws]
    plan.close()
    assert np.all(np.isfinite(grads[0])) and np.abs(grads[0]).max() > 0
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, c, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    gk = dec["gauss"]
    okeys = (gk["sigma"], gk["qidx"], gk["pidx"])
    plus = okeys[0] == 1
    assert set(zip(okeys[1][plus].tolist(), okeys[2][plus].tolist())) == keys
    dirs = [_smooth_direction_3d(prob.n, 1)]
    for f in np.argsort(-np.abs(grads[0].ravel()))[:2]:
        e = np.zeros(prob.n)
        e.ravel()[f] = 1.0
        dirs.append(e)
    worst = 0.0
    for v in dirs:
        _, jv = O.frozen_set_traces_tangent(g, c, v, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box,
                                            okeys, prob.nsteps, prob.dt, REC, prob.kappa, xr)
        for w, gr in zip(ws, grads):
            lhs = float(np.sum(gr * v))
            rhs = float(np.sum(w[0] * jv.real))
            err = abs(lhs - rhs) / (np.linalg.norm(w) * np.linalg.norm(jv.real))
            worst = max(worst, err)
            assert err <= 1e-12, (lhs, rhs, err)
    print("3D adjoint vs oracle tangent, worst relative difference %.3e" % worst)
