"""torch.autograd.Function over ddelm_solve / ddelm_backward.

u = DDELMSolve.apply(solver, f_int, g_bnd) returns the network values at the
evaluation points; its backward calls the library's adjoint (ddelm_backward),
which reuses the setup's factorisations.  Gradients flow to the forcing
values f_int and the Dirichlet values g_bnd (the map is linear in both).

u = DDELMSolveScaled.apply(solver, f_int, g_bnd, scale) also takes the
hidden-layer scale s as a 0-d tensor (equal to the solver's problem scale);
its gradient dL/ds comes from the same ddelm_backward call (the library's
reverse-mode scale gradient at the forward solve), with no further setup.
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
        return u

    @staticmethod
    def backward(ctx, grad_u):
        if ctx.needs_input_grad[3]:
            gf, gg, _, gs = ctx.solver.backward(grad_u=grad_u.contiguous(), scale=True)
            return None, gf, gg, torch.tensor(gs, dtype=grad_u.dtype, device=grad_u.device)
        gf, gg, _ = ctx.solver.backward(grad_u=grad_u.contiguous())
        return None, gf, gg, None


def solve_u_scaled(solver, f_int, g_bnd, scale):
    return DDELMSolveScaled.apply(solver, f_int, g_bnd, scale)
