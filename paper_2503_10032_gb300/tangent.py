"""Derivative of the DDELM-NN solution with respect to the hidden-layer scale s
(w = s w_hat, b = s b_hat, Sec. 2.2).

Forward mode.  The interface unknowns solve r(mu, s) = b_theta(s) -
S_theta(s) mu = 0 (Eq. (nn-mixed)) and u = u(mu, s) is the reconstruction of
Eq. (coarse_sol_2) at the evaluation points, so

    dmu/ds = S_theta^{-1} dr/ds|_mu,    du/ds = du/ds|_mu + (du/dmu) dmu/ds.

The tangent solve and du/dmu (the linear part of the reconstruction: the
residual call with zero data) use the base setup's factors on the GPU.  The
partial derivatives at fixed mu are central differences of two setups at
s (1 +- h): the residual and the reconstruction at a fixed mu involve no
iteration, so their differences carry no solver noise and h = 1e-6 leaves
about 1e-9 relative error (truncation h^2, rounding ~1e-16 / h).
"""
from __future__ import annotations

import dataclasses


def scale_tangent(solver, f_int, g_bnd, rel_step=1e-6):
    """(u, du/ds) at the evaluation points for the solver's problem and data (f, g)."""
    from .ddelm import Solver
    torch = solver.torch
    prob = solver.prob
    c, mu_full, u, info, rc = solver.solve(f_int, g_bnd)
    n_pi = solver.sizes.n_pi
    mu = mu_full[n_pi:].contiguous()
    h = rel_step * prob.scale
    res = []
    for sign in (1.0, -1.0):
        other = Solver(dataclasses.replace(prob, scale=prob.scale + sign * h), device=solver.device,
                       stream=solver.stream, **solver.opt_kw)
        r_s, _, u_s = other.interface_residual(f_int, g_bnd, mu)
        res.append((r_s.clone(), u_s.clone()))
        other.close()
    dr = (res[0][0] - res[1][0]) / (2.0 * h)
    du_mu = (res[0][1] - res[1][1]) / (2.0 * h)
    mudot, _ = solver.interface_solve(dr)
    zf = torch.zeros_like(f_int)
    zg = torch.zeros_like(g_bnd)
    _, _, u_lin = solver.interface_residual(zf, zg, mudot)
    return u, du_mu + u_lin
