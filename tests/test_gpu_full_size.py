"""Parity with the oracle at the full sizes of the two 2D workloads the path is quoted on.

* The lens workload as specified: 256 x 256 on [0,1)^2, c = 1 + 0.3 exp(-|x - (.5,.5)|^2/0.02),
  eps = 1/256, q-stride 8, box 192 (more than one 128-wide p tile per q), tau = 1e-3,
  kappa = 6, T = 0.5 (500 RK4 steps through the lens). psi+ element by element against
  the oracle's FFT route, the selected set outside its guard band, 300 sampled rays at
  T, and the field on a ragged 64 x 64 subgrid, where the oracle propagates every kept
  Gaussian of both branches and sums them term by term: FP64 path <= 1e-10, mixed path
  (tensor-core FBI stage 2 and reconstruction) <= 1e-4.
* The benchmark's layered workload (737 x 241, 15 Hz ring at 10 m depth, eps from
  15 Hz, s = 5, box 128, kappa = 6) over its whole time, T = 2 s, with the 20 000 largest
  |psi+| per branch so that the oracle can propagate every Gaussian: the field on a
  ragged subgrid, FP64 <= 1e-10.
"""

import functools

import numpy as np
import pytest

import oracle as O
import test_gpu_parity as TP
from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


def _subgrid(prob, step, offset):
    """Points of a regular subgrid (every step-th point from offset on each axis)."""
    axes = [prob.origin[k] + prob.h[k] * np.arange(offset[k], prob.n[k], step)
            for k in range(prob.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    flat = np.ravel_multi_index(tuple(np.meshgrid(
        *[np.arange(offset[k], prob.n[k], step) for k in range(prob.dim)], indexing="ij")),
        prob.n).ravel()
    return np.stack([m.ravel() for m in mesh], axis=1), flat


@functools.lru_cache(maxsize=1)
def _lens_oracle():
    prob = WL.lens_2d()  # 256^2, eps = 1/256, s = 8, box = 192, tau = 1e-3, kappa = 6, T = 0.5
    assert prob.n == (256, 256) and prob.shots[0].box == (192, 192) and prob.nsteps == 500
    sh = prob.shots[0]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau,
                      q_subset=TP.active_q(prob, sh))
    x, flat = _subgrid(prob, 4, (1, 3))
    uo = TP.oracle_field(prob, 0, dec, x)
    assert np.linalg.norm(uo.imag) <= 1e-12 * np.linalg.norm(uo.real)
    return prob, dec, flat, uo.real


def test_lens_workload_fp64_against_oracle():
    prob, dec, flat, uo = _lens_oracle()
    plan, counts, u = TP.run_gpu(prob)
    qi, pi = TP.check_decomposition(plan, prob, dec)
    assert counts[0] == qi.size and counts[0] > 50_000
    gs = dec["gauss"]
    plus = np.flatnonzero(gs["sigma"] == 1)
    pick = np.random.default_rng(21).choice(plus, 300, replace=False)
    TP.check_rays(plan, prob, 0, gs["qidx"][pick], gs["pidx"][pick], tol_q=1e-9, tol_a=1e-9)
    err = TP.rel(u[0].ravel()[flat], uo)
    print("lens 256^2, T = 0.5: %d Gaussians, field rel-L2 vs oracle %.3e" % (counts[0], err))
    assert err <= TP.FIELD_TOL, err
    plan.close()


def test_lens_workload_mixed_against_oracle():
    import torch

    prob, dec, flat, uo = _lens_oracle()
    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               precision=F.FGA_MIXED_TF32X3)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    plan.reconstruct(out)
    plan.sync()
    plan.close()
    err = TP.rel(out[0].cpu().numpy().ravel()[flat], uo)
    print("lens 256^2, T = 0.5, mixed: field rel-L2 vs oracle %.3e" % err)
    assert err <= MIXED_TOL, err


def test_layered_full_time_field_against_oracle():
    prob = WL.layered_single().with_(keep_n=20_000)  # T = 2 s, 2000 steps
    assert prob.nsteps == 2000
    plan, counts, u = TP.run_gpu(prob)
    assert counts[0] == 20_000
    sh = prob.shots[0]
    g = O.Grid(prob.n, prob.h, prob.origin, prob.periodic)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, prob.tau,
                      keep_n=prob.keep_n, q_subset=TP.active_q(prob, sh))
    TP.check_decomposition(plan, prob, dec)
    x, flat = _subgrid(prob, 5, (2, 1))
    uo = TP.oracle_field(prob, 0, dec, x)
    err = TP.rel(u[0].ravel()[flat], uo.real)
    print("layered, T = 2 s, 20000 largest: field rel-L2 vs oracle %.3e" % err)
    assert err <= TP.FIELD_TOL, err
    plan.close()
