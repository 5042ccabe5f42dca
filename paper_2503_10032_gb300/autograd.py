"""torch.autograd.Function over ddelm_solve / ddelm_backward.

u = DDELMSolve.apply(solver, f_int, g_bnd) returns the network values at the
evaluation points; its backward calls the library's adjoint (ddelm_backward),
which reuses the setup's factorisations.  Gradients flow to the forcing
values f_int and the Dirichlet values g_bnd (the map is linear in both).
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
