"""N-largest selection (keep_n > 0, the selection of the paper's experiment): per shot the
keep_n largest |psi+| over the valid (q, p), ties by q index then p index, against the
oracle's selection; and the field of the whole pipeline with it against the oracle."""

import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_1304_3542_gb300 import workloads as WL
from test_gpu_parity import FIELD_TOL, _grid, oracle_field, rel, run_gpu

pytestmark = pytest.mark.gpu


def _problem(keep_n, N=96, nshots=1):
    prob = WL.lens_2d(N=N, eps=1.0 / 400 * (96 / N) ** 2, T=0.05, dt=1e-3, s=2, box=64,
                      tau=0.0, k0=30 * math.pi * N / 96, width2=0.004 * (96 / N) ** 2,
                      x0=(0.45, 0.3))
    return dataclasses.replace(prob, keep_n=keep_n)


@pytest.mark.parametrize("keep_n", [6, 48, 521, 5650])
def test_keep_n_set_matches_oracle(keep_n):
    prob = _problem(keep_n)
    plan, counts, u = run_gpu(prob)
    sh = prob.shots[0]
    g = _grid(prob)
    dec = O.decompose(g, prob.velocity, sh.u0, sh.u1, sh.eps, sh.q_stride, sh.box, 0.0,
                      keep_n=keep_n)
    assert counts[0] == keep_n
    gs = dec["gauss"]
    plus = gs["sigma"] == 1
    okeys = set(zip(gs["qidx"][plus].tolist(), gs["pidx"][plus].tolist()))
    qi, pi, _ = plan.gaussians(0)
    gkeys = set(zip(qi.tolist(), pi.tolist()))
    # entries may trade places only where |psi+| equals the cut to within rounding
    a = np.abs(dec["psi_plus"])
    rows = {int(r): i for i, r in enumerate(dec["rows"])}
    cut = min(a[rows[q], p] for q, p in okeys)
    for q, p in gkeys ^ okeys:
        assert abs(a[rows[q], p] - cut) <= 1e-12 * cut, (q, p)
    # the + set is the keep_n largest: every kept |psi+| >= every dropped valid one
    kept = np.array([a[rows[q], p] for q, p in gkeys])
    assert kept.min() >= cut * (1 - 1e-12)
    uo = oracle_field(prob, 0, dec, prob.grid_points())
    assert rel(u[0].ravel(), uo.real) <= FIELD_TOL
    plan.close()


def test_keep_n_more_than_available_takes_all_valid():
    prob = _problem(10 ** 9)
    plan, counts, _ = run_gpu(prob)
    tau0 = dataclasses.replace(prob, keep_n=0, tau=0.0)
    plan0, counts0, _ = run_gpu(tau0)
    assert counts[0] == counts0[0]
    qa, pa, _ = plan.gaussians(0)
    qb, pb, _ = plan0.gaussians(0)
    assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
    plan.close()
    plan0.close()


def test_keep_n_per_shot_in_a_batch():
    full = WL.layered_batch(nshots=3, T=0.02)
    prob = dataclasses.replace(full, keep_n=5650, tau=0.0)
    plan, counts, _ = run_gpu(prob, integrate_exited=False)
    assert list(counts) == [5650] * 3
    for s in range(3):
        single = dataclasses.replace(prob, shots=[prob.shots[s]])
        p1, c1, _ = run_gpu(single, integrate_exited=False)
        qa, pa, _ = plan.gaussians(s)
        qb, pb, _ = p1.gaussians(0)
        assert np.array_equal(qa, qb) and np.array_equal(pa, pb)
        p1.close()
    plan.close()
