"""Differentiable RK stepping: torch.autograd.Function over dg_rk_step /
dg_rk_step_adjoint.

Forward: n_steps unlimited RK steps with a frozen timestep, keeping one
checkpoint of the state per step.  Backward: for every step in reverse, the
library recomputes the stage states from the checkpoint and applies the
exact transpose of the step (dg_rk_step_adjoint).
"""
import torch


class RKSteps(torch.autograd.Function):
    """W_N = step^N(W_0) with a frozen dt; gradients with respect to W_0."""

    @staticmethod
    def forward(ctx, W0, solver, n_steps, dt):
        if dt <= 0:
            raise ValueError("RKSteps needs a frozen timestep dt > 0")
        W = W0.detach().clone()
        ckpts = []
        for _ in range(int(n_steps)):
            ckpts.append(W.clone())
            solver.rk_step(W, dt)
        ctx.solver, ctx.dt, ctx.ckpts = solver, float(dt), ckpts
        return W

    @staticmethod
    def backward(ctx, grad_out):
        lam = grad_out.detach().to(ctx.solver.dtype).contiguous().clone()
        for Wn in reversed(ctx.ckpts):
            ctx.solver.rk_step_adjoint(Wn, ctx.dt, lam, out=lam)
        ctx.ckpts = None
        return lam, None, None, None


def rk_steps(W0, solver, n_steps, dt):
    return RKSteps.apply(W0, solver, n_steps, dt)
