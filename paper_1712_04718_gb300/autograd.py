"""The SE k-space energy as a differentiable PyTorch function.

E^L(x, q) (Sec. 1 Eq. 1.6, computed by the SE method of Sec. 3) is returned
as a 0-d float64 tensor.  Its backward pass is the adjoint kernel of libse
(se_adjoint): with the upstream gradient g = dl/dE,

    dl/dx = -g F    (F = -dE/dx, the analytic force of Sec. 3.1)
    dl/dq =  g phi  (E = 1/2 q^T A q, so dE/dq = A q = phi)

The forward pass runs spread and scale (no gather: only the energy is
needed); the backward pass gathers from the grid that forward left in the
plan.  If the plan has evaluated anything else in between, or recompute=True
(memory-tight use: nothing is kept for backward but the inputs), backward
first recomputes the spread and the scaling.
"""
import torch

from .se import Plan


class SEEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, q, plan, recompute):
        # the scaling step writes E (an empty system writes nothing)
        E = (torch.empty if plan.N > 0 else torch.zeros)(1, dtype=torch.float64,
                                                          device=xyz.device)
        plan.spread(xyz, q)
        plan.scale(E)
        ctx.save_for_backward(xyz, q)
        ctx.plan = plan
        ctx.generation = plan.generation
        ctx.recompute = bool(recompute)
        return E[0]

    @staticmethod
    def backward(ctx, gE):
        xyz, q = ctx.saved_tensors
        plan = ctx.plan
        if ctx.recompute or plan.generation != ctx.generation:
            plan.spread(xyz, q)
            plan.scale(None)
        g = gE.detach()
        if g.dtype != torch.float64 or g.dim() != 1:
            g = g.to(torch.float64).reshape(1).contiguous()
        gx = torch.empty_like(xyz) if ctx.needs_input_grad[0] else None
        gq = torch.empty_like(q) if ctx.needs_input_grad[1] else None
        plan.adjoint(xyz, q, g, gx, gq)
        return gx, gq, None, None


def se_energy(xyz, q, plan: Plan, recompute=False):
    """E^L of charges q at positions xyz (CUDA tensors of the plan's dtype);
    differentiable in xyz and q."""
    return SEEnergy.apply(xyz, q, plan, recompute)
