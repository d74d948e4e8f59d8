"""torch.autograd.Function over the library: the impacts Imp_i(theta, r) of Eq. 4 under the policy
that L Sinkhorn iterations (Problem (7)) produce for the per-item cost c_uik = -r(u,i) e_k
exp(theta_i), differentiated by the library's gradient kernels.

The forward pass loads r and theta into a `FairRank` problem (FR_PARAM_ITEM), solves every consumer
and returns Imp (float64, on theta's device). The backward pass hands dLoss/dImp to `fr_grad`
as omega, so one kernel launch per consumer batch returns both dLoss/dtheta and dLoss/dr. With
grad_mode FR_GRAD_UNROLLED that is the exact derivative of the L-iteration map (the reverse sweep
of the adjoint kernel); with FR_GRAD_IMPLICIT it is the derivative at the Sinkhorn fixed point.

A problem holds one solve: a backward pass must follow its own forward pass before the next
forward pass on the same problem, otherwise it raises.
"""
from __future__ import annotations

import torch

from . import fairrank as fr


class SinkhornImpact(torch.autograd.Function):
    """imp = SinkhornImpact.apply(theta, r, problem) with theta [n_items], r [n_users, n_items]
    (float32 or bfloat16 matching the problem's relevance storage) on the problem's device."""

    @staticmethod
    def forward(ctx, theta, r, problem):
        if problem.param != fr.PARAM_ITEM:
            raise ValueError("SinkhornImpact needs a FR_PARAM_ITEM problem")
        if theta.shape != (problem.I,) or r.shape != (problem.U, problem.I):
            raise ValueError(f"theta must be ({problem.I},) and r ({problem.U}, {problem.I})")
        problem.set_relevance(r.detach().contiguous())
        problem.set_state(param=theta.detach().to(torch.float32).contiguous())
        imp, _, _ = problem.impacts()
        version = getattr(problem, "_autograd_version", 0) + 1
        problem._autograd_version = version
        ctx.problem, ctx.version = problem, version
        ctx.theta_dtype, ctx.r_dtype = theta.dtype, r.dtype
        return torch.from_numpy(imp).to(theta.device)

    @staticmethod
    def backward(ctx, g_imp):
        p = ctx.problem
        if getattr(p, "_autograd_version", None) != ctx.version:
            raise RuntimeError("the problem was re-solved since this forward pass")
        omega = g_imp.detach().to(device="cuda", dtype=torch.float32).contiguous()
        want_dr = bool(ctx.needs_input_grad[1])
        out = p.grad(omega=omega, want_dr=want_dr, device=True)
        dth, dr = out if want_dr else (out, None)
        dth = dth.to(ctx.theta_dtype) if ctx.needs_input_grad[0] else None
        if dr is not None:
            dr = dr.to(ctx.r_dtype)
        return dth, dr, None


def sinkhorn_impact(theta, r, problem):
    """Functional form of SinkhornImpact.apply."""
    return SinkhornImpact.apply(theta, r, problem)
