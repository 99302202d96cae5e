"""torch.autograd Functions over the device solver (argument marshalling only).

The parameters theta are a float64 tensor (g^2 Nc, G(x_G)^{-1}) or
(g^2 Nc, G(x_G)^{-1}, Z(x_Z)^{-1}); the last defaults to the plan's value.  Every
forward and backward pass runs in the CUDA kernels behind include/dse.h:

  Residual      F(c; theta)                 backward: dse_vjp (v^T dF/dc without the
                                            Newton matrix) and dse_param_derivatives
  ImplicitSolve c*(theta) with F(c*, theta) = 0 (dse_solve)
                                            backward: J(c*)^T lambda = dL/dc*
                                            (dse_adjoint_solve), dL/dtheta =
                                            -lambda^T dF/dtheta
  Dressing      ln G(x), ln Z(x) at momenta x (dse_dressing)
                                            backward: dse_dressing_vjp

The residual is the renormalised ghost-gluon system of arXiv:1206.1779 Sec. 2-3;
the implicit-function gradient is the adjoint of its Newton system.
"""
from __future__ import annotations

import torch

from ._binding import Plan


def _apply_theta(plan: Plan, theta: torch.Tensor) -> None:
    vals = [float(v) for v in theta.detach().cpu().tolist()]
    if len(vals) not in (2, 3):
        raise ValueError("theta must hold (g2nc, ginv_G) or (g2nc, ginv_G, zinv_Z)")
    zinv = vals[2] if len(vals) == 3 else plan.params["zinv_Z"]
    plan.set_couplings(vals[0], vals[1], zinv)


def _theta_grad(w: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    return w[: theta.numel()].to(device=theta.device, dtype=theta.dtype).reshape(theta.shape)


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, coeffs: torch.Tensor, theta: torch.Tensor):
        _apply_theta(plan, theta)
        c = coeffs.detach().contiguous()
        F = plan.residual(c)
        ctx.plan = plan
        ctx.save_for_backward(c, theta.detach())
        return F

    @staticmethod
    def backward(ctx, gF):
        c, theta = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        v = gF.detach().contiguous()
        gc = plan.vjp(c, v) if ctx.needs_input_grad[1] else None
        gt = _theta_grad(plan.param_vjp(c, v), theta) if ctx.needs_input_grad[2] else None
        return None, gc, gt


class ImplicitSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, theta: torch.Tensor, c0: torch.Tensor, tol: float = 1e-10, max_iter: int = 50,
                rho_relax: float = 1.0, n_relax: int = 0):
        _apply_theta(plan, theta)
        c = c0.detach().clone().contiguous()
        it, _ = plan.solve(c, tol=tol, max_iter=max_iter, rho_relax=rho_relax, n_relax=n_relax)
        ctx.plan = plan
        ctx.iterations = it
        ctx.save_for_backward(c, theta.detach())
        return c

    @staticmethod
    def backward(ctx, gc):
        c, theta = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        lam, _ = plan.adjoint_solve(c, gc.detach().contiguous())
        gt = -_theta_grad(plan.param_vjp(c, lam), theta) if ctx.needs_input_grad[1] else None
        return None, gt, None, None, None, None, None


class Dressing(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan: Plan, coeffs: torch.Tensor, theta: torch.Tensor, x: torch.Tensor):
        _apply_theta(plan, theta)
        x = x.detach().contiguous()
        lG, lZ = plan.dressing(coeffs.detach().contiguous(), x)
        ctx.plan = plan
        ctx.save_for_backward(x, theta.detach())
        return lG, lZ

    @staticmethod
    def backward(ctx, gG, gZ):
        x, theta = ctx.saved_tensors
        plan = ctx.plan
        _apply_theta(plan, theta)
        gG = torch.zeros_like(x) if gG is None else gG.detach().contiguous()
        gZ = torch.zeros_like(x) if gZ is None else gZ.detach().contiguous()
        wg = torch.zeros(3, dtype=torch.float64, device=x.device)
        gc = plan.dressing_vjp(x, gG, gZ, out_g2nc=wg)
        gt = _theta_grad(wg, theta) if ctx.needs_input_grad[2] else None
        return None, gc if ctx.needs_input_grad[1] else None, gt, None


def residual(plan: Plan, coeffs: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    return Residual.apply(plan, coeffs, theta)


def solve(plan: Plan, theta: torch.Tensor, c0: torch.Tensor, tol: float = 1e-10, max_iter: int = 50,
          rho_relax: float = 1.0, n_relax: int = 0) -> torch.Tensor:
    return ImplicitSolve.apply(plan, theta, c0, tol, max_iter, rho_relax, n_relax)


def dressing(plan: Plan, coeffs: torch.Tensor, theta: torch.Tensor, x: torch.Tensor):
    return Dressing.apply(plan, coeffs, theta, x)
