"""torch.autograd wrapper: FRKC2 steps as a differentiable function of (u0, kappa).

The forward runs ``frkc2_adjoint_forward`` (the integration, keeping a checkpoint every
``ckpt_every`` steps and the last segment's stage tape in a workspace saved for backward);
the backward runs ``frkc2_adjoint_backward`` (per-segment stage recompute and the reverse
stage replay) and returns dJ/du0 and, for a conductivity field, dJ/dkappa.  Both run in the
CUDA library; this module only allocates the workspaces and passes pointers.
"""
from __future__ import annotations

import torch

from . import frkc2 as F


class FRKC2Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, kappa, plan, ndim, bc, precision, dx, dt, nsteps, ckpt_every):
        n = tuple(reversed(u0.shape))
        u0 = u0.detach().contiguous()
        kappa = kappa.detach().contiguous()
        prob = F.make_problem(ndim, n, dx, bc, "field", precision, kappa_field=kappa)
        ws = torch.empty(F.frkc2_adjoint_workspace_size(plan, prob, nsteps, ckpt_every),
                         dtype=torch.uint8, device=u0.device)
        F.frkc2_workspace_reset(ws)
        u = torch.empty_like(u0)
        F.frkc2_adjoint_forward(plan, prob, dt, nsteps, ckpt_every, u0, u, ws)
        ctx.save_for_backward(kappa)
        ctx.ws = ws
        ctx.shape = u0.shape
        ctx.state_dtype = u0.dtype
        ctx.cfg = (plan, ndim, bc, precision, dx, dt, nsteps, ckpt_every)
        return u

    @staticmethod
    def backward(ctx, g):
        (kappa,) = ctx.saved_tensors
        plan, ndim, bc, precision, dx, dt, nsteps, ckpt_every = ctx.cfg
        n = tuple(reversed(ctx.shape))
        prob = F.make_problem(ndim, n, dx, bc, "field", precision, kappa_field=kappa)
        du0 = torch.empty(ctx.shape, dtype=ctx.state_dtype, device=kappa.device)
        dk = torch.empty_like(kappa) if ctx.needs_input_grad[1] else None
        F.frkc2_adjoint_backward(plan, prob, dt, nsteps, ckpt_every, g.contiguous().to(ctx.state_dtype),
                                 du0, dk, ctx.ws)
        ctx.ws = None
        return du0, dk, None, None, None, None, None, None, None, None


def frkc2_steps(u0, kappa, plan, dt, nsteps, bc="periodic", precision=None, dx=1.0, ckpt_every=8):
    """Differentiable FRKC2 integration of div(kappa grad u) for a conductivity field.

    u0, kappa: CUDA tensors of the grid shape (numpy order, last axis x); double for FP64,
    float state and kappa for FP32, double state and float kappa for MIXED.
    """
    if precision is None:
        precision = "fp64" if u0.dtype == torch.float64 else "fp32"
    return FRKC2Steps.apply(u0, kappa, plan, u0.dim(), bc, precision, dx, dt, nsteps, ckpt_every)
