"""fga_run_graph: propagate + reconstruct captured once as a CUDA graph and replayed.

The replay runs the same kernels on the same buffers, and the field reduction has a
fixed order, so every replay must give the eager result bit for bit; receiver traces
are summed with atomics (in an order that changes from run to run), so they agree to
rounding of sums with cancellation: 1e-11 of the largest trace value. The graph is captured again when the
receivers or the output buffer change."""

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _problem(N=96, T=0.05):
    return WL.lens_2d(N=N, eps=1.0 / 400 * (96 / N) ** 2, T=T, dt=1e-3, s=2, box=64,
                      tau=1e-3, kappa=6.0, k0=24 * np.pi, width2=0.004)


def _eager(prob, precision, stream):
    import torch

    plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
    u0, u1 = F.stacked_initial_data(prob)
    out = torch.zeros((len(prob.shots),) + prob.n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
        plan.propagate()
        plan.reconstruct(out)
    plan.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", [F.FGA_FP64, F.FGA_MIXED_TF32X3])
def test_replay_matches_eager(precision):
    import torch

    prob = _problem()
    stream = torch.cuda.Stream()
    ref = _eager(prob, precision, stream)
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
    u0, u1 = F.stacked_initial_data(prob)
    with torch.cuda.stream(stream):
        a, b = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
        plan.decompose(a, b)
        outs = [torch.full((len(prob.shots),) + prob.n, np.nan, dtype=torch.float64,
                           device="cuda") for _ in range(2)]
        results = []
        for out in (outs[0], outs[0], outs[0], outs[1], outs[1]):
            out.fill_(np.nan)
            plan.run_graph(out)
            plan.sync()
            results.append(out.cpu().numpy())
    assert np.abs(ref).max() > 0
    for r in results:
        assert np.array_equal(r, ref)


def test_replay_traces_and_receiver_change():
    import torch

    prob = _problem(N=64, T=0.1)
    stream = torch.cuda.Stream()
    xr = np.stack([np.linspace(0.2, 0.8, 13), np.full(13, 0.55)], axis=1)
    plan = F.plan_from_problem(prob, stream=stream.cuda_stream)
    u0, u1 = F.stacked_initial_data(prob)
    out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
        plan.set_receivers(xr, 5)
        plan.propagate()
        plan.reconstruct(out)
        plan.sync()
        tr_eager = plan.traces().copy()
        u_eager = out.cpu().numpy()
        for _ in range(3):
            plan.run_graph(out)
            plan.sync()
            assert np.array_equal(out.cpu().numpy(), u_eager)
            tr = plan.traces()
            scale = np.abs(tr_eager).max()
            assert scale > 0
            assert np.abs(tr - tr_eager).max() <= 1e-11 * scale
        # new receivers: the graph must be captured again around the new buffers
        plan.set_receivers(xr[::2], 1)
        plan.run_graph(out)
        plan.sync()
        tr2 = plan.traces()
        plan.propagate()
        plan.sync()
        tr2_eager = plan.traces()
    assert tr2.shape == tr2_eager.shape and tr2.shape != tr_eager.shape
    assert np.abs(tr2 - tr2_eager).max() <= 1e-11 * np.abs(tr2_eager).max()


def test_default_stream_rejected():
    import torch

    prob = _problem(N=64, T=0.02)
    plan = F.plan_from_problem(prob, stream=None)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FGAError) as ei:
        plan.run_graph(out)
    assert ei.value.status == F.FGA_ERR_INVALID
    with pytest.raises(F.FGAError):
        plan.run_graph(np.zeros((1,) + prob.n))


@pytest.mark.parametrize("precision", [F.FGA_FP64, F.FGA_MIXED_TF32X3])
def test_autotune_choice_and_results(precision):
    """The autotuner's choice is one of its candidates, leaves every ray state unchanged
    (bit for bit) and the field unchanged up to the order of the partial sums; a plan
    given the same choice reproduces the tuned field bit for bit."""
    import torch

    prob = _problem(N=128, T=0.05)
    stream = torch.cuda.Stream()
    u0, u1 = F.stacked_initial_data(prob)
    shape = (len(prob.shots),) + prob.n

    def fresh():
        plan = F.plan_from_problem(prob, stream=stream.cuda_stream, precision=precision)
        with torch.cuda.stream(stream):
            plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
        return plan

    with torch.cuda.stream(stream):
        ref_plan = fresh()
        ref = torch.zeros(shape, dtype=torch.float64, device="cuda")
        ref_plan.propagate()
        ref_plan.reconstruct(ref)
        ref_plan.sync()
        ref_state = ref_plan.state(0)
        tuned_plan = fresh()
        out = torch.zeros(shape, dtype=torch.float64, device="cuda")
        per_sm, seg, variant = tuned_plan.autotune(out)
        tuned_plan.sync()
    assert tuned_plan.tuning() == (per_sm, seg, variant)
    assert 1 <= per_sm <= 64 and variant in (0, 1)
    base = 128 if precision == F.FGA_MIXED_TF32X3 else 256
    assert seg in [base << k for k in range(5)]  # a small case: no raise for memory
    st = tuned_plan.state(0)
    for k in ref_state:
        assert np.array_equal(st[k], ref_state[k]), k
    u_ref, u_tuned = ref.cpu().numpy(), out.cpu().numpy()
    # FP64: sums in another order. Mixed precision: each work item's partial tile is an
    # FP32 accumulation in tensor memory whose rounding grows with the segment length, so
    # two segment lengths differ by up to the mixed form's own error against the FP64
    # path, which the precision policy bounds by 1e-4
    tol = 1e-13 if precision == F.FGA_FP64 else 1e-4
    assert np.linalg.norm(u_tuned - u_ref) <= tol * np.linalg.norm(u_ref)
    with torch.cuda.stream(stream):
        again = fresh()
        again.set_tuning(per_sm, seg, variant)
        out2 = torch.zeros(shape, dtype=torch.float64, device="cuda")
        again.propagate()
        again.reconstruct(out2)
        again.sync()
    assert np.array_equal(out2.cpu().numpy(), u_tuned)
    with pytest.raises(F.FGAError):
        again.set_tuning(-1, 0)
    with pytest.raises(F.FGAError):
        again.set_tuning(2, 1 << 21)
    with pytest.raises(F.FGAError):
        again.set_tuning(2, 1024, 2)


def test_ray_kernel_variants_give_identical_states():
    """The two register budgets of the 2D ray kernel (255 and 168 registers per thread)
    integrate every ray bit for bit alike, at full occupancy and at one block per SM."""
    import torch

    prob = _problem(N=96, T=0.05)
    u0, u1 = F.stacked_initial_data(prob)
    ref = None
    for variant in (0, 1):
        for per_sm in (0, 1):
            plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream)
            plan.set_tuning(per_sm, 0, variant)
            plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
            plan.propagate()
            plan.sync()
            st = plan.state(0)
            plan.close()
            if ref is None:
                ref = st
            else:
                for k in ref:
                    assert np.array_equal(st[k], ref[k]), (variant, per_sm, k)
