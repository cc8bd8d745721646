"""torch.autograd.Functions over libfga: traces at receivers, or the wavefield at time T,
as a function of the velocity.

FGATraces: forward(velocity) runs decompose -> propagate (with receivers) and returns the
traces [nshots][nrec][nrx]; backward(grad_traces) calls fga_grad, the hand-written
discrete adjoint, and returns d loss / d velocity on the grid.

FGAField: forward(velocity) returns u(T) of Eq. recons on the whole grid [nshots][n...],
recorded by putting a receiver on every grid point and recording once, at T; backward is
the same adjoint with the residual at that record (the adjoint of the reconstruction sum
and of the rays behind it).

The set of Gaussians is the one selected by the forward call (held fixed for the
derivative). Velocity and outputs are float64 CUDA tensors; PyTorch only supplies memory
and the stream.

The forward's plan (its device memory holds the checkpoints the backward needs) lives
until the backward has run, or until the autograd graph that holds it is freed (the
plan's finaliser destroys it); a forward that cannot be differentiated (grad mode off,
or a velocity that does not require grad) destroys it at once.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fga as F


class FGATraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, velocity, prob, receivers, record_every, precision=F.FGA_FP64,
                integrate_exited=False, interp=F.FGA_BSPLINE_APPROX, keep_plan=True):
        plan = F.plan_from_problem(prob, velocity=velocity.detach().contiguous(),
                                   stream=torch.cuda.current_stream().cuda_stream,
                                   precision=precision, integrate_exited=integrate_exited,
                                   interp=interp)
        plan.set_receivers(receivers, record_every)
        u0, u1 = F.stacked_initial_data(prob)
        plan.decompose(torch.from_numpy(u0).to(velocity.device),
                       torch.from_numpy(u1).to(velocity.device))
        plan.propagate()
        nrec = prob.nsteps // record_every + 1
        out = torch.empty((len(prob.shots), nrec, len(receivers)), dtype=torch.float64,
                          device=velocity.device)
        plan.traces(out)
        if not keep_plan:
            plan.close()
            plan = None
        ctx.plan = plan
        ctx.shape = velocity.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        grad = torch.empty(ctx.shape, dtype=torch.float64, device=grad_out.device)
        ctx.plan.grad(grad_out.contiguous(), grad)
        ctx.plan.close()
        ctx.plan = None
        return grad, None, None, None, None, None, None, None


def _differentiable(velocity):
    return torch.is_grad_enabled() and velocity.requires_grad


def traces(velocity, prob, receivers, record_every, **kw):
    return FGATraces.apply(velocity, prob, receivers, record_every,
                           kw.get("precision", F.FGA_FP64), kw.get("integrate_exited", False),
                           kw.get("interp", F.FGA_BSPLINE_APPROX), _differentiable(velocity))


def grid_receivers(prob):
    """Every grid point as a receiver [npts][dim], C order. The last point of each axis is
    moved 2 ulps inwards so that it passes the inside-the-grid check however the host
    compiler rounds the grid's end point; the field there changes by ~1e-16 relative."""
    axes = []
    for k in range(prob.dim):
        x = prob.origin[k] + prob.h[k] * np.arange(prob.n[k], dtype=np.float64)
        x[-1] = np.nextafter(np.nextafter(x[-1], -np.inf), -np.inf)
        axes.append(x)
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([m.ravel() for m in mesh], axis=1))


class FGAField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, velocity, prob, precision=F.FGA_FP64, integrate_exited=False,
                interp=F.FGA_BSPLINE_APPROX, keep_plan=True):
        plan = F.plan_from_problem(prob, velocity=velocity.detach().contiguous(),
                                   stream=torch.cuda.current_stream().cuda_stream,
                                   precision=precision, integrate_exited=integrate_exited,
                                   interp=interp)
        xr = grid_receivers(prob)
        plan.set_receivers(xr, prob.nsteps)  # records at t = 0 and t = T
        u0, u1 = F.stacked_initial_data(prob)
        plan.decompose(torch.from_numpy(u0).to(velocity.device),
                       torch.from_numpy(u1).to(velocity.device))
        plan.propagate()
        ns = len(prob.shots)
        tr = torch.empty((ns, 2, xr.shape[0]), dtype=torch.float64, device=velocity.device)
        plan.traces(tr)
        if not keep_plan:
            plan.close()
            plan = None
        ctx.plan = plan
        ctx.shape = velocity.shape
        ctx.ns, ctx.npts = ns, xr.shape[0]
        return tr[:, 1].reshape((ns,) + tuple(prob.n)).contiguous()

    @staticmethod
    def backward(ctx, grad_out):
        res = torch.zeros((ctx.ns, 2, ctx.npts), dtype=torch.float64, device=grad_out.device)
        res[:, 1] = grad_out.reshape(ctx.ns, ctx.npts)
        grad = torch.empty(ctx.shape, dtype=torch.float64, device=grad_out.device)
        ctx.plan.grad(res, grad)
        ctx.plan.close()
        ctx.plan = None
        return grad, None, None, None, None, None


def field(velocity, prob, **kw):
    """u(T) on the grid [nshots][n...], differentiable in the velocity (1D and 2D, open
    axes)."""
    return FGAField.apply(velocity, prob, kw.get("precision", F.FGA_FP64),
                          kw.get("integrate_exited", False),
                          kw.get("interp", F.FGA_BSPLINE_APPROX), _differentiable(velocity))
