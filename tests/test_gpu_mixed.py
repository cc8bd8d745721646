"""Mixed-precision reconstruction (tensor cores, split TF32 factors, FP32 accumulation,
FP64 phase anchors) against the FP64 path: rel-L2 <= 1e-4 on the field."""

import math

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


def _field(prob, precision):
    import torch

    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               precision=precision)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    out = torch.zeros((len(prob.shots),) + prob.n, dtype=torch.float64, device="cuda")
    plan.reconstruct(out)
    plan.sync()
    plan.close()
    return out.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prob", [
    WL.lens_2d(N=150, eps=1.0 / 976, T=0.05, dt=1e-3, s=2, box=64, tau=1e-3,
               k0=30 * math.pi * 150 / 96, width2=0.004 * (96 / 150) ** 2, x0=(0.45, 0.3)),
    WL.layered_single(),
], ids=["lens_150_ragged", "layered_T2"])
def test_mixed_matches_fp64(prob):
    u64 = _field(prob, F.FGA_FP64)
    umx = _field(prob, F.FGA_MIXED_TF32X3)
    err = _rel(umx, u64)
    assert err <= MIXED_TOL, err


def test_mixed_batched_shots():
    prob = WL.layered_batch(nshots=3, T=0.1)
    u64 = _field(prob, F.FGA_FP64)
    umx = _field(prob, F.FGA_MIXED_TF32X3)
    for s in range(3):
        assert _rel(umx[s], u64[s]) <= MIXED_TOL
