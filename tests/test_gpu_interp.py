"""FGA_BSPLINE_INTERP: the plan turns the velocity samples into the spline coefficients with
the interpolating prefilter (fga_spline_prefilter, checked against the oracle's dense
solve on the CPU in test_abi.py), and fga_grad maps dJ/dC back to the samples with the
same symmetric map.

On the GPU a plan given samples c with FGA_BSPLINE_INTERP must compute what a plan given
the coefficients C = prefilter(c) with FGA_BSPLINE_APPROX computes: the same field (bit
for bit: identical coefficients, deterministic kernels), the same traces (to the last
bits of their atomic sums), and the gradient prefilter(dJ/dC) of the other plan's.
"""

import math

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _problem():
    return WL.lens_2d(N=64, eps=1.0 / 400, T=0.05, dt=1e-3, s=2, box=32, tau=1e-2, kappa=8.0,
                      k0=24 * math.pi, width2=0.004, x0=(0.4937, 0.3), center=(0.5071, 0.4963))


def _run(prob, velocity, interp):
    import torch

    plan = F.plan_from_problem(prob, velocity=np.ascontiguousarray(velocity),
                               stream=torch.cuda.current_stream().cuda_stream,
                               integrate_exited=True, interp=interp)
    x = np.linspace(0.15, 0.85, 29)
    plan.set_receivers(np.stack([x, np.full_like(x, 0.5)], axis=1), 5)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    u = plan.reconstruct()
    tr = plan.traces()
    g = plan.grad(np.ascontiguousarray(tr))
    plan.close()
    return u, tr, g


def test_interp_plan_equals_approx_plan_on_prefiltered_coefficients():
    prob = _problem()
    c = prob.velocity
    C = F.spline_prefilter(c, prob.periodic)
    assert C.min() > 0.0 and np.max(np.abs(C - c)) > 1e-6
    uA, trA, gA = _run(prob, c, F.FGA_BSPLINE_INTERP)
    uB, trB, gB = _run(prob, C, F.FGA_BSPLINE_APPROX)
    assert np.array_equal(uA, uB)
    assert np.linalg.norm(trA - trB) <= 1e-12 * np.linalg.norm(trB)
    ref = F.spline_prefilter(gB, prob.periodic)
    assert np.linalg.norm(gA - ref) <= 1e-10 * np.linalg.norm(ref)
