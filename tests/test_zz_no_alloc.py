"""fga_reconstruct_static: the reconstruction for callers that cannot allocate device
memory (code where cudaMalloc is off limits, or whose device memory is all budgeted)
keeps its scratch in a fixed device array and must give the field that the
plan-based fga_reconstruct gives, call after call (the array keeps the previous
call's contents, so every call has to clear what must start at zero).

This file is collected last on purpose; it passes alone in a fresh process too.
"""

import math

import numpy as np
import pytest

from paper_1304_3542_gb300 import fga as F
from paper_1304_3542_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-10


def _plan_field_and_terms(prob):
    """Run the plan-based path; return its field and the Gaussians' rows and coefficients
    coef = 2 W a psi (2 pi eps)^{-3d/2} exp(i S/eps) of shot 0, on the device."""
    import torch

    plan = F.plan_from_problem(prob, stream=torch.cuda.current_stream().cuda_stream)
    u0, u1 = F.stacked_initial_data(prob)
    plan.decompose(torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda())
    plan.propagate()
    ref = torch.zeros((1,) + prob.n, dtype=torch.float64, device="cuda")
    plan.reconstruct(ref)
    plan.sync()
    st = plan.state(0)
    _, _, psi = plan.gaussians(0)
    plan.close()
    sh = prob.shots[0]
    d = prob.dim
    W = 1.0
    for k in range(d):
        W *= sh.q_stride[k] * prob.h[k] * 2 * math.pi * sh.eps / (sh.box[k] * prob.h[k])
    coef = (2 * W * st["a"] * psi * (2 * math.pi * sh.eps) ** (-1.5 * d)
            * np.exp(1j * st["S"] / sh.eps))
    qp = np.ascontiguousarray(np.concatenate([st["Q"].T, st["P"].T], axis=0))
    cf = np.ascontiguousarray(np.stack([coef.real, coef.imag], axis=1))
    return (ref[0].cpu().numpy(), torch.from_numpy(qp).cuda(), torch.from_numpy(cf).cuda())


def _static(prob, qp, cf, fill=np.nan):
    import torch

    u = torch.full(prob.n, fill, dtype=torch.float64, device="cuda")
    F.reconstruct_static(prob.dim, prob.n, prob.h, prob.origin, prob.periodic,
                         prob.shots[0].eps, prob.kappa, qp, cf, u,
                         stream=torch.cuda.current_stream().cuda_stream)
    return u.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_reconstruction_matches_the_plan_call_after_call():
    cases = [
        # 710k Gaussians: several chunks through the fixed tile-list array
        WL.layered_single(T=0.05),
        # a smaller 2D grid with a ragged tile edge
        WL.lens_2d(N=96, eps=1.0 / 400, T=0.05, dt=1e-3, s=2, box=64, tau=1e-3,
                   k0=30 * math.pi, width2=0.004, x0=(0.45, 0.3)),
        # 1D periodic: images of the window on both sides
        WL.periodic_1d(),
    ]
    for prob in cases:
        ref, qp, cf = _plan_field_and_terms(prob)
        first = _static(prob, qp, cf)
        second = _static(prob, qp, cf, fill=1e300)  # same call again on a dirty output
        assert _rel(first, ref) <= FIELD_TOL, prob.name
        assert _rel(second, ref) <= FIELD_TOL, prob.name
        assert np.array_equal(first, second)


def test_static_reconstruction_rejects_oversized_grids():
    import torch

    n = (64 * 129, 64 * 128)  # 16512 tiles of 64 x 64: more than the fixed array holds
    # a buffer of the grid's full size (541 MB), so that no order of the checks in the
    # library can make the call touch memory outside it
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    qp = torch.zeros((4, 1), dtype=torch.float64, device="cuda")
    cf = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FGAError) as ei:
        F.reconstruct_static(2, n, (0.01, 0.01), (0.0, 0.0), (False, False), 1e-3, 6.0, qp, cf, u)
    assert ei.value.status == 7  # FGA_ERR_CAPACITY
    assert "tiles" in str(ei.value)
    del u
    torch.cuda.empty_cache()


def test_static_reconstruction_wrapper_checks_buffer_sizes():
    """The Python binding refuses buffers whose sizes do not match (the C entry point
    cannot see sizes); nothing is launched."""
    import torch

    n = (64, 64)
    qp = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    cf = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        F.reconstruct_static(2, n, (0.01, 0.01), (0.0, 0.0), (False, False), 1e-3, 6.0, qp, cf,
                             torch.zeros(64 * 63, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        F.reconstruct_static(2, n, (0.01, 0.01), (0.0, 0.0), (False, False), 1e-3, 6.0, qp,
                             cf[:2], torch.zeros(n, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        F.reconstruct_static(2, n, (0.01, 0.01), (0.0, 0.0), (False, False), 1e-3, 6.0,
                             qp.reshape(-1)[:11], cf, torch.zeros(n, dtype=torch.float64,
                                                                  device="cuda"))
