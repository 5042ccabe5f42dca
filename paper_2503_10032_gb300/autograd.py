"""torch.autograd.Function over ddelm_solve / ddelm_backward.

u = DDELMSolve.apply(solver, f_int, g_bnd) returns the network values at the
evaluation points; its backward calls the library's adjoint (ddelm_backward),
which reuses the setup's factorisations.  Gradients flow to the forcing
values f_int and the Dirichlet values g_bnd (the map is linear in both).

u = DDELMSolveScaled.apply(solver, f_int, g_bnd, scale) also takes the
hidden-layer scale s as a 0-d tensor (equal to the solver's problem scale);
its gradient is <dL/du, du/ds> with du/ds from the forward-mode tangent of
`tangent.scale_tangent`.
"""
from __future__ import annotations

import torch


class DDELMSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, f_int, g_bnd):
        c, mu, u, info, rc = solver.solve(f_int.detach(), g_bnd.detach())
        ctx.solver = solver
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        gf, gg, _ = ctx.solver.backward(grad_u=grad_u.contiguous())
        return None, gf, gg


def solve_u(solver, f_int, g_bnd):
    return DDELMSolve.apply(solver, f_int, g_bnd)


class DDELMSolveScaled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, f_int, g_bnd, scale):
        if abs(float(scale) - float(solver.prob.scale)) > 1e-12 * abs(float(solver.prob.scale)):
            raise ValueError("scale must equal the solver's problem scale")
        c, mu, u, info, rc = solver.solve(f_int.detach(), g_bnd.detach())
        ctx.solver = solver
        ctx.save_for_backward(f_int.detach(), g_bnd.detach())
        return u

    @staticmethod
    def backward(ctx, grad_u):
        from .tangent import scale_tangent
        f, g = ctx.saved_tensors
        gf, gg, _ = ctx.solver.backward(grad_u=grad_u.contiguous())
        gs = None
        if ctx.needs_input_grad[3]:
            _, du_ds = scale_tangent(ctx.solver, f, g)
            gs = (grad_u * du_ds).sum()
        return None, gf, gg, gs


def solve_u_scaled(solver, f_int, g_bnd, scale):
    return DDELMSolveScaled.apply(solver, f_int, g_bnd, scale)
