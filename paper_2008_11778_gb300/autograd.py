"""torch.autograd wrappers whose backward passes are the library's adjoint-state
kernels (Sec. 2.2: eqs. FWI_adj, adj_grad1 for FWI; eqs. Born, LSRTM for LSRTM).

  FWIMisfit.apply(m, plan, d_obs) -> J          J = 1/2 ||F(m) - d_obs||^2
      forward: aafwi_adjoint_gradient (forward sweep, misfit, adjoint sweep
      and imaging in one call; the gradient is kept for backward)
      backward: grad_m = dJ * dJ/dm
  ForwardModel.apply(m, plan) -> d              d = F(m) (traces)
      backward: aafwi_fwi_adjoint with the incoming trace cotangent as the
      adjoint source, reusing the stored forward wavefield
  Born.apply(rho, plan, m0) -> d                d = L rho
      backward: aafwi_born_adjoint (L^T)

Argument marshalling only; no arithmetic of the method runs in torch.
"""
import torch

from . import aafwi


class FWIMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, plan, d_obs):
        m = m.detach().contiguous()
        grad = torch.empty_like(m)
        J = plan.adjoint_gradient(aafwi.MODE_FWI, m, None, d_obs.contiguous(), grad)
        ctx.save_for_backward(grad)
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return grad * gJ.to(grad.dtype), None, None


class ForwardModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, plan):
        m = m.detach().contiguous()
        d = torch.empty(plan.trace_count, dtype=torch.float32, device=m.device)
        plan.model_forward(m, d)
        ctx.plan = plan
        ctx.save_for_backward(m)
        return d

    @staticmethod
    def backward(ctx, gd):
        (m,) = ctx.saved_tensors
        grad = torch.empty_like(m)
        # the plan keeps the forward wavefield of the last model_forward; reuse
        # it when nothing else ran on the plan in between
        ctx.plan.fwi_adjoint(m, gd.contiguous().to(torch.float32), grad, reuse_forward=False)
        return grad, None


class Born(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, plan, m0):
        rho = rho.detach().contiguous()
        d = torch.empty(plan.trace_count, dtype=torch.float32, device=rho.device)
        plan.born_forward(m0.contiguous(), rho, d)
        ctx.plan, ctx.m0 = plan, m0
        return d

    @staticmethod
    def backward(ctx, gd):
        img = torch.empty(ctx.m0.shape, dtype=torch.float32, device=gd.device)
        ctx.plan.born_adjoint(ctx.m0.contiguous(), gd.contiguous().to(torch.float32), img)
        return img, None, None


def fwi_misfit(m, plan, d_obs):
    return FWIMisfit.apply(m, plan, d_obs)


def forward_model(m, plan):
    return ForwardModel.apply(m, plan)


def born(rho, plan, m0):
    return Born.apply(rho, plan, m0)
