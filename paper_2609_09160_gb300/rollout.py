"""Differentiable rollout: gradients of a loss on the state after T steps with respect to the
per-site body-force field and the initial moments, by the hand-written adjoint kernel of the
library with checkpoint-and-recompute (the paper has no adjoint; this is the discrete adjoint of
the library's own step).

Forward: T steps from M0, storing the internal state every K steps (ceil(T/K)+1 checkpoints).
Backward: for each segment, newest first, the K states are recomputed from the segment's
checkpoint into a (K+1)-state buffer, then lbf_adjoint_step runs from the segment's last step to
its first, carrying lambda = dL/dM and accumulating dL/dF in FP64.
Memory: (ceil(T/K) + K + 2) internal states plus two lambda buffers, instead of T states.
"""
import math

import torch

from .solver import Solver


class Rollout(torch.autograd.Function):
    """M_T = Rollout.apply(force_field, M0, solver, steps, K).

    `force_field` must be the tensor the solver was created with (the library reads it by
    pointer); `solver` must be single-component with 'f32' or 'f64' storage. The returned public
    state M_T has the solver's compute dtype; the gradient flows to force_field and M0.
    The FP64 force gradient is also left in solver.grad_force64.
    """

    @staticmethod
    def forward(ctx, force_field, M0, solver, steps, K):
        if not isinstance(solver, Solver) or solver.force_field is None:
            raise ValueError("Rollout needs a Solver created with force_field")
        if force_field.data_ptr() != solver.force_field.data_ptr():
            raise ValueError("force_field must be the tensor the solver was created with")
        steps, K = int(steps), int(K)
        nseg = max(1, math.ceil(steps / K))
        solver.set_moments(M0.detach())
        ckpt = solver.new_state(count=nseg + 1)
        solver.copy_state(ckpt[0])
        done = 0
        for j in range(nseg):
            n = min(K, steps - done)
            solver.step(n)
            done += n
            solver.copy_state(ckpt[j + 1])
        MT = solver.moments(dtype=solver.compute_dtype)
        ctx.solver, ctx.steps, ctx.K, ctx.nseg = solver, steps, K, nseg
        ctx.m0_dtype = M0.dtype
        ctx.save_for_backward(ckpt)
        return MT

    @staticmethod
    def backward(ctx, grad_MT):
        (ckpt,) = ctx.saved_tensors
        solver, steps, K, nseg = ctx.solver, ctx.steps, ctx.K, ctx.nseg
        cdt = solver.compute_dtype
        lam = grad_MT.detach().to(dtype=cdt).contiguous().clone()
        lam_b = torch.empty_like(lam)
        gF = torch.zeros((3,) + solver.shape, dtype=torch.float64, device=solver.device)
        seg = solver.new_state(count=K + 1)
        seg.copy_(ckpt[0].expand_as(seg))  # solid sites never change: every slot starts valid
        for j in reversed(range(nseg)):
            t0 = j * K
            n = min(K, steps - t0)
            seg[0].copy_(ckpt[j])
            for k in range(n):
                solver.step_state(seg[k], seg[k + 1])
            for k in reversed(range(n)):
                solver.adjoint_step(seg[k], seg[k + 1], lam, lam_b, gF)
                lam, lam_b = lam_b, lam
        solver.grad_force64 = gF
        return gF.to(solver.force_field.dtype), lam.to(ctx.m0_dtype), None, None, None


def rollout(force_field, M0, solver, steps, K=50):
    return Rollout.apply(force_field, M0, solver, steps, K)
