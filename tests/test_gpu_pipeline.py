"""fga_run_pipeline: decompose + propagate + reconstruct of every shot as one captured
CUDA graph, with the Gaussian counts computed and used on the device.

* A replay gives the eager three-step result bit for bit (the rays do not depend on
  their order, the binning and the field reduction have fixed orders), call after
  call, in FP64 and in the mixed precision, for one shot and for a batch of shots.
* Replayed on new data with the same support, the graph selects, propagates and sums
  the new data's own Gaussians: the field equals a fresh eager plan's bit for bit and
  fga_count reports the new counts (read back from the device).
* Data that need more Gaussians than the capacities the graph was captured with, or
  whose support gives other active q rectangles, are reported as FGA_ERR_CAPACITY by
  the next fga_sync (the replay stays inside its buffers).
"""

import math

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _lens(N=96, T=0.04):
    return WL.lens_2d(N=N, eps=1.0 / 400 * (96 / N) ** 2, T=T, dt=1e-3, s=2, box=64,
                      tau=1e-3, kappa=6.0, k0=24 * math.pi, width2=0.004)


def _eager(prob, u0, u1, precision, stream):
    import torch

    plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
    out = torch.zeros((len(prob.shots),) + prob.n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
        plan.propagate()
        plan.reconstruct(out)
    plan.sync()
    counts = [plan.count(s) for s in range(len(prob.shots))]
    plan.close()
    return out.cpu().numpy(), counts


@pytest.mark.parametrize("which", ["lens_fp64", "lens_mixed", "batch3_fp64", "batch3_mixed"])
def test_replay_matches_eager_bitwise(which):
    import torch

    prob = _lens() if which.startswith("lens") else WL.layered_batch(nshots=3, T=0.03)
    precision = F.FGA_MIXED_TF32X3 if which.endswith("mixed") else F.FGA_FP64
    stream = torch.cuda.Stream()
    u0, u1 = F.stacked_initial_data(prob)
    ref, ref_counts = _eager(prob, u0, u1, precision, stream)
    assert np.abs(ref).max() > 0
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
    with torch.cuda.stream(stream):
        a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
        out = torch.full((len(prob.shots),) + prob.n, np.nan, dtype=torch.float64, device="cuda")
        for _ in range(4):  # the first call runs eagerly and captures; then replays
            out.fill_(np.nan)
            plan.run_pipeline(a, b, out)
            plan.sync()
            assert np.array_equal(out.cpu().numpy(), ref)
            assert [plan.count(s) for s in range(len(prob.shots))] == ref_counts
    plan.close()


def test_replay_selects_the_new_data_gaussians():
    import torch

    prob = _lens()
    stream = torch.cuda.Stream()
    u0, u1 = F.stacked_initial_data(prob)
    # same support, other values: the branch split mixes psi0 and psi1 differently
    v0, v1 = np.ascontiguousarray(1.1 * u0), np.ascontiguousarray(0.6 * u1)
    ref_a, counts_a = _eager(prob, u0, u1, F.FGA_FP64, stream)
    ref_b, counts_b = _eager(prob, v0, v1, F.FGA_FP64, stream)
    assert counts_a != counts_b
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
        out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
        plan.run_pipeline(a, b, out)  # captured on the first data
        plan.sync()
        assert np.array_equal(out.cpu().numpy(), ref_a)
        for src, ref, counts in ((np.stack([v0, v1]), ref_b, counts_b),
                                 (np.stack([u0, u1]), ref_a, counts_a),
                                 (np.stack([v0, v1]), ref_b, counts_b)):
            a.copy_(torch.from_numpy(src[0]))
            b.copy_(torch.from_numpy(src[1]))
            plan.run_pipeline(a, b, out)  # the same graph, replayed
            plan.sync()
            assert np.array_equal(out.cpu().numpy(), ref)
            assert [plan.count(0)] == counts
    plan.close()


def test_too_many_gaussians_are_reported():
    import torch

    prob = _lens()
    stream = torch.cuda.Stream()
    u0, u1 = F.stacked_initial_data(prob)
    rng = np.random.default_rng(4)
    # the same support (the packet is nonzero on the whole grid) with a broadband part:
    # far more (q, p) pass the threshold than the graph was sized for
    w0 = np.ascontiguousarray(u0 + 0.3 * np.abs(u0).max() * rng.standard_normal(u0.shape))
    _, counts_a = _eager(prob, u0, u1, F.FGA_FP64, stream)
    _, counts_w = _eager(prob, w0, u1, F.FGA_FP64, stream)
    assert counts_w[0] > 1.25 * counts_a[0] + 1024
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
        out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
        plan.run_pipeline(a, b, out)
        plan.sync()
        a.copy_(torch.from_numpy(w0))
        plan.run_pipeline(a, b, out)
        with pytest.raises(F.FGAError) as ei:
            plan.sync()
    assert ei.value.status == F.FGA_ERR_CAPACITY
    plan.close()
    # a fresh plan handles the new data
    ref_w, cw = _eager(prob, w0, u1, F.FGA_FP64, stream)
    assert cw == counts_w and np.isfinite(ref_w).all()


def test_other_support_is_reported():
    import torch

    prob = WL.layered_single(T=0.01)
    stream = torch.cuda.Stream()
    u0, u1 = F.stacked_initial_data(prob)
    # the same ring 2.5 km further along x: same eps (the top layer is uniform), other
    # active q rectangle
    s0, s1 = (np.ascontiguousarray(np.roll(x, 200, axis=1)) for x in (u0, u1))
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
        out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
        plan.run_pipeline(a, b, out)
        plan.sync()
        a.copy_(torch.from_numpy(s0))
        b.copy_(torch.from_numpy(s1))
        plan.run_pipeline(a, b, out)
        with pytest.raises(F.FGAError) as ei:
            plan.sync()
    assert ei.value.status == F.FGA_ERR_CAPACITY
    assert "support" in str(ei.value)
    plan.close()


def test_pipeline_rejects_what_it_cannot_capture():
    import torch

    prob = _lens(N=64, T=0.01)
    u0, u1 = F.stacked_initial_data(prob)
    a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
    out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    plan = F.plan_from_problem(prob, stream=None)  # the legacy default stream
    with pytest.raises(F.FGAError) as ei:
        plan.run_pipeline(a, b, out)
    assert ei.value.status == F.FGA_ERR_INVALID
    plan.close()
    stream = torch.cuda.Stream()
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    with pytest.raises(F.FGAError) as ei:
        plan.run_pipeline(u0, u1, out)  # host inputs
    assert ei.value.status == F.FGA_ERR_INVALID
    plan.close()
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    plan.set_receivers(np.array([[0.5, 0.5]]), 5)
    with pytest.raises(F.FGAError) as ei:
        plan.run_pipeline(a, b, out)
    assert ei.value.status == F.FGA_ERR_INVALID
    plan.close()
