"""The bounded waits of the tensor-core kernels give up cleanly (failure detection
without a GPU fault).

With a wait budget of 0 polls every in-loop completion wait of FBI stage 2 and of the
reconstruction gives up at once: the CTA stops issuing MMAs, waits for its single
outstanding commit with the default budget, releases its tensor memory and sets the
status word. The next fga_sync reports FGA_ERR_TIMEOUT and marks the plan failed; the
context stays usable, and a fresh plan on the same data gives the normal result.
"""

import math

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _prob():
    return WL.lens_2d(N=96, eps=1.0 / 400, T=0.02, dt=1e-3, s=2, box=64, tau=1e-3,
                      k0=30 * math.pi, width2=0.004, x0=(0.45, 0.3))


def _run(prob, tries=None):
    import torch

    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               precision=F.FGA_MIXED_TF32X3)
    if tries is not None:
        plan.set_wait_budget(tries)
    u0, u1 = F.stacked_initial_data(prob)
    out = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    plan.reconstruct(out)
    return plan, out


def test_wait_budget_zero_reports_timeout_and_a_fresh_plan_works():
    import torch

    prob = _prob()
    ref_plan, ref = _run(prob)
    ref_plan.sync()
    ref = ref.cpu().numpy()
    ref_plan.close()
    plan, _ = _run(prob, tries=0)
    with pytest.raises(F.FGAError) as ei:
        plan.sync()
    assert ei.value.status == F.FGA_ERR_TIMEOUT
    with pytest.raises(F.FGAError) as ei:  # the plan is marked failed
        plan.propagate()
    assert ei.value.status == F.FGA_ERR_STATE
    plan.close()
    torch.cuda.synchronize()  # the context is still usable
    again, out = _run(prob, tries=-1)
    again.sync()
    assert np.array_equal(out.cpu().numpy(), ref)
    again.close()


def test_wait_budget_rejects_out_of_range():
    prob = _prob()
    plan = F.plan_from_problem(prob)
    with pytest.raises(F.FGAError) as ei:
        plan.set_wait_budget(1 << 33)
    assert ei.value.status == F.FGA_ERR_INVALID
    plan.set_wait_budget(1000)
    plan.set_wait_budget(-1)
    plan.close()
