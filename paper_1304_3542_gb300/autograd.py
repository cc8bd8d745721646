"""torch.autograd.Function over libfga: traces at receivers as a function of the velocity.

forward(velocity) runs decompose -> propagate (with receivers) and returns the traces
[nshots][nrec][nrx]; backward(grad_traces) calls fga_grad, the hand-written discrete
adjoint, and returns d loss / d velocity on the grid. The set of Gaussians is the one
selected by the forward call (held fixed for the derivative). Velocity and traces are
float64 CUDA tensors; PyTorch only supplies memory and the stream.
"""

from __future__ import annotations

import torch

from . import fga as F


class FGATraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, velocity, prob, receivers, record_every, precision=F.FGA_FP64,
                integrate_exited=False):
        plan = F.plan_from_problem(prob, velocity=velocity.detach().contiguous(),
                                   stream=torch.cuda.current_stream().cuda_stream,
                                   precision=precision, integrate_exited=integrate_exited)
        plan.set_receivers(receivers, record_every)
        u0, u1 = F.stacked_initial_data(prob)
        plan.decompose(torch.from_numpy(u0).to(velocity.device),
                       torch.from_numpy(u1).to(velocity.device))
        plan.propagate()
        nrec = prob.nsteps // record_every + 1
        out = torch.empty((len(prob.shots), nrec, len(receivers)), dtype=torch.float64,
                          device=velocity.device)
        plan.traces(out)
        ctx.plan = plan
        ctx.shape = velocity.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        grad = torch.empty(ctx.shape, dtype=torch.float64, device=grad_out.device)
        ctx.plan.grad(grad_out.contiguous(), grad)
        ctx.plan.close()
        return grad, None, None, None, None, None


def traces(velocity, prob, receivers, record_every, **kw):
    return FGATraces.apply(velocity, prob, receivers, record_every,
                           kw.get("precision", F.FGA_FP64), kw.get("integrate_exited", False))
