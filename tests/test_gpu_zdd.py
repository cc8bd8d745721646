"""FGA_Z_DIVIDED: d_zQ and d_zP by central divided differences across auxiliary rays
started at (q +- dq e_k, p) and (q, p +- dp e_k) (the alternative to Eqs. dzQ, dzP named
after Eq. op_zZ), against the oracle's propagate_dd.

* Ray states (Q, P, a and the difference quotients A, B) of a sample of the oracle's
  Gaussians, element by element, and the field against the oracle's field built from its
  own divided-difference rays (both branches literally), on the 2D lens with full and
  ragged tiles and on the 1D periodic problem (whose auxiliary rays cross the period).
* As the offsets shrink, the GPU field approaches the dynamic-ray field at second order.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _grid(prob):
    return O.Grid(prob.n, prob.h, prob.origin, prob.periodic)


def _lens(N):
    return WL.lens_2d(N=N, eps=1.0 / 400 * (96 / N) ** 2, T=0.05, dt=1e-3, s=2, box=64,
                      tau=1e-3, k0=30 * math.pi * N / 96, width2=0.004 * (96 / N) ** 2,
                      x0=(0.45, 0.3))


def _run(prob, z_method, eta):
    import torch

    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True, z_method=z_method, dz_eta=eta)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    u = plan.reconstruct()[0]
    plan.sync()
    return plan, u


def _offsets(prob, eta):
    sh = prob.shots[0]
    dq = [eta * sh.q_stride[k] * prob.h[k] for k in range(prob.dim)]
    dp = [eta * 2.0 * math.pi * sh.eps / (sh.box[k] * prob.h[k]) for k in range(prob.dim)]
    return dq, dp


def _check(prob, eta, field_tol):
    plan, u = _run(prob, F.FGA_Z_DIVIDED, eta)
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau)
    gs = dec["gauss"]
    dq, dp = _offsets(prob, eta)
    ost = O.propagate_dd(g, prob.velocity, prob.nsteps, prob.dt, gs["sigma"], gs["q"], gs["p"],
                         dq, dp)
    # ray states of a sample of the + branch, found in the GPU's list by their keys
    qi, pi, _ = plan.gaussians(0)
    pos = {k: i for i, k in enumerate(zip(qi.tolist(), pi.tolist()))}
    plus = np.flatnonzero(gs["sigma"] == 1)[::41]
    idx = np.array([pos[(int(gs["qidx"][j]), int(gs["pidx"][j]))] for j in plus])
    st = plan.state(0)
    dQ = st["Q"][idx] - ost["Q"][plus]
    for k in range(prob.dim):
        if prob.periodic[k]:
            L = prob.n[k] * prob.h[k]
            dQ[:, k] -= L * np.round(dQ[:, k] / L)
    assert np.max(np.abs(dQ)) <= 1e-12 * max(1.0, np.max(np.abs(ost["Q"])))
    assert np.max(np.abs(st["P"][idx] - ost["P"][plus])) <= 1e-12 * max(1.0, np.max(np.abs(ost["P"])))
    assert np.max(np.abs(st["a"][idx] - ost["a"][plus]) / np.abs(ost["a"][plus])) <= 1e-9
    amax = max(1.0, float(np.max(np.abs(ost["A"]))), float(np.max(np.abs(ost["B"]))))
    assert np.max(np.abs(st["A"][idx] - ost["A"][plus])) <= 1e-9 * amax
    assert np.max(np.abs(st["B"][idx] - ost["B"][plus])) <= 1e-9 * amax
    # the field, both branches literally on the oracle side
    W = O.quadrature_weight(g, sh.eps, sh.q_stride, sh.box)
    uo = O.reconstruct(g, sh.eps, prob.kappa, W, ost["Q"], ost["P"], ost["a"], gs["psi"], ost["S"],
                       prob.grid_points())
    err = np.linalg.norm(u.ravel() - uo.real) / np.linalg.norm(uo.real)
    plan.close()
    assert err <= field_tol, err


@pytest.mark.parametrize("N", [96, 150])
def test_divided_differences_match_the_oracle_2d(N):
    _check(_lens(N), 0.1, 1e-9)


def test_divided_differences_match_the_oracle_1d_periodic():
    _check(WL.periodic_1d(T=0.05), 0.5, 1e-9)


def test_divided_differences_converge_to_dynamic_rays():
    prob = _lens(96)
    _, u_dyn = _run(prob, F.FGA_Z_DYNAMIC, 0.0)
    diffs = []
    for eta in (0.4, 0.2, 0.1):
        plan, u = _run(prob, F.FGA_Z_DIVIDED, eta)
        plan.close()
        diffs.append(np.linalg.norm(u - u_dyn) / np.linalg.norm(u_dyn))
    assert diffs[-1] <= 1e-4, diffs
    for e0, e1 in zip(diffs, diffs[1:]):
        assert 2.5 <= e0 / e1 <= 4.5, diffs
