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


def _psi(prob, precision):
    import torch

    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream,
                               precision=precision)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.sync()
    psi, _ = plan.psi(0)
    qi, pi, _ = plan.gaussians(0)
    plan.close()
    return psi, set(zip(qi.tolist(), pi.tolist()))


@pytest.mark.parametrize("prob", [
    WL.lens_2d(N=150, eps=1.0 / 976, T=0.05, dt=1e-3, s=2, box=64, tau=1e-3,
               k0=30 * math.pi * 150 / 96, width2=0.004 * (96 / 150) ** 2, x0=(0.45, 0.3)),
    WL.lens_2d(N=256, T=0.01),
    WL.layered_single(T=0.01),
], ids=["lens_150_box64", "lens_256_box192", "layered_box128"])
def test_mixed_fbi_matches_fp64(prob):
    """Stage 2 of the FBI on the tensor cores (split TF32, FP32 accumulation, one or more
    128 x 128 tiles of p per q): psi+ within 1e-5 of max |psi+| of the FP64 transform
    (FP32 sums over K = 2 n_b terms, n_b up to 192), and the same Gaussian set up to the
    Gaussians whose |psi+| lies within twice that margin of the threshold."""
    p64, k64 = _psi(prob, F.FGA_FP64)
    pmx, kmx = _psi(prob, F.FGA_MIXED_TF32X3)
    scale = np.abs(p64).max()
    err = np.abs(pmx - p64).max() / scale
    assert err <= 1e-5, err
    a = np.abs(p64)
    thr = prob.tau * scale
    for q, pj in k64 ^ kmx:
        assert abs(a[q, pj] - thr) <= 2e-5 * scale, (q, pj, a[q, pj], thr)
