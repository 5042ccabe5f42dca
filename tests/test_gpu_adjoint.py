"""Adjoint (ddelm_backward) against the forward solve, the oracle and finite
differences; gradients of a solution loss w.r.t. Fourier forcing coefficients."""
import numpy as np
import pytest

from oracle import ddelm as odd
from paper_2503_10032_gb300 import inputs
from parity_util import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_10032_gb300 import build
    build.build()
    from paper_2503_10032_gb300 import ddelm
    return ddelm


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_is_transpose_of_solve(D, prec):
    """<c_bar, L(df, dg)> == <L^T c_bar, (df, dg)> and L^T c_bar == J^T c_bar of the oracle."""
    p = inputs.small_problem(3, 2, M=16, n_int=40, edge_pts=3, n_rhs=1, seed=8)
    kw = dict(eps_rel=1e-6, tol=1e-12, precision=D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED)
    s = D.Solver(p, **kw)
    rng = np.random.default_rng(0)
    nI, nB = p.f_int.shape[0], p.g_bnd.shape[0]
    cbar = rng.standard_normal((int(p.M.sum()), 1))
    ubar = rng.standard_normal((int(p.n_eval.sum()), 1))
    df, dg = rng.standard_normal((nI, 1)), rng.standard_normal((nB, 1))
    c, mu, u, info, rc = s.solve(_t(df), _t(dg))
    gf, gg, binfo = s.backward(grad_c=_t(cbar), grad_u=_t(ubar))
    lhs = float((cbar * c.cpu().numpy()).sum() + (ubar * u.cpu().numpy()).sum())
    rhs = float((gf.cpu().numpy() * df).sum() + (gg.cpu().numpy() * dg).sum())
    assert abs(lhs - rhs) <= 1e-8 * max(abs(lhs), 1.0)
    # oracle Jacobian of (f, g) -> (c, u) by solving for every unit vector at once
    q = inputs.small_problem(3, 2, M=16, n_int=40, edge_pts=3, n_rhs=1, seed=8)
    n = nI + nB
    q.f_int = np.hstack([np.eye(nI), np.zeros((nI, nB))])
    q.g_bnd = np.hstack([np.zeros((nB, nI)), np.eye(nB)])
    ref = odd.solve(q, odd.Options(eps_rel=1e-6))
    Jc = np.concatenate(ref["c"])            # [sum M, n]
    Ju = ref["u_eval"]                       # [sum n_eval, n]
    g_ref = Jc.T @ cbar + Ju.T @ ubar        # [n, 1]
    g_gpu = np.vstack([gf.cpu().numpy(), gg.cpu().numpy()])
    assert g_gpu.shape == (n, 1)
    assert close(g_gpu, g_ref, (1e-6 if prec == "fp64" else 1e-5), "g_gpu vs g_ref")


def test_fourier_coefficient_gradient(D):
    """Loss = mean (u - sin(pi x) sin(pi y))^2 over the evaluation points, forcing
    f = sum_{p,q<=4} a_pq sin(p pi x) sin(q pi y), g = 0: gradient w.r.t. a by the
    adjoint, by central finite differences and by the oracle's linear map."""
    import torch
    from paper_2503_10032_gb300.autograd import solve_u
    rng = np.random.default_rng(4)
    a0 = rng.standard_normal(16)
    p = inputs.make_problem(3, 3, 40, 120, 4, scale=8.0, init="paper", seed=41,
                            solutions=[inputs.fourier_forcing(a0)], n_eval=16)
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12)
    X, Y = p.x_int[:, 0], p.x_int[:, 1]
    basis = np.stack([np.sin((i + 1) * np.pi * X) * np.sin((j + 1) * np.pi * Y) for i in range(4) for j in range(4)], 1)
    Bt = _t(basis)
    ut = _t(np.sin(np.pi * p.x_eval[:, 0]) * np.sin(np.pi * p.x_eval[:, 1]))[:, None]
    g = torch.zeros((p.g_bnd.shape[0], 1), dtype=torch.float64, device="cuda")

    def loss_of(a):
        f = Bt @ a[:, None]
        u = solve_u(s, f, g)
        return ((u - ut) ** 2).mean()

    a = torch.tensor(a0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss_of(a)
    L.backward()
    grad = a.grad.cpu().numpy()
    # central differences (the map a -> u is linear: exact up to roundoff)
    h = 1e-3
    fd = np.zeros(16)
    with torch.no_grad():
        for k in range(16):
            e = torch.zeros(16, dtype=torch.float64, device="cuda")
            e[k] = h
            fd[k] = (float(loss_of(a + e)) - float(loss_of(a - e))) / (2 * h)
    assert close(grad, fd, 1e-6, "grad vs fd")
    # oracle: u is linear in a; du/da_pq = solve(basis column pq, g = 0)
    q = inputs.make_problem(3, 3, 40, 120, 4, scale=8.0, init="paper", seed=41,
                            solutions=[inputs.fourier_forcing(a0)], n_eval=16)
    q.f_int = basis
    q.g_bnd = np.zeros((p.g_bnd.shape[0], 16))
    ref = odd.solve(q, odd.Options(eps_rel=1e-6))
    U = ref["u_eval"]                          # [n_eval, 16]
    u_now = U @ a0
    grad_ref = 2.0 / len(u_now) * U.T @ (u_now - np.sin(np.pi * p.x_eval[:, 0]) * np.sin(np.pi * p.x_eval[:, 1]))
    assert close(grad, grad_ref, 1e-6, "grad vs grad_ref")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_scale_gradient(D, prec):
    """dL/ds for the hidden-layer scale s (w = s w_hat, b = s b_hat) from one
    ddelm_backward call (the library's reverse mode at the solve, no further
    setup), against a fourth-order central difference of the FP64 oracle's
    solution, for three losses: the squared error of u against
    sin(pi x) sin(pi y) (through torch.autograd), a seeded linear functional of
    u, and a seeded linear functional of the coefficients c."""
    import dataclasses
    import torch
    from paper_2503_10032_gb300.autograd import solve_u_scaled
    p = inputs.make_problem(3, 3, 40, 120, 4, scale=8.0, init="paper", seed=43,
                            solutions=[inputs._sin2pix_cos3piy()], n_eval=16)
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12, precision=pr)
    f = _t(p.f_int)
    g = _t(p.g_bnd)
    target = np.sin(np.pi * p.x_eval[:, 0]) * np.sin(np.pi * p.x_eval[:, 1])
    wu = inputs.interface_vectors(len(target), 1, 1, 11)[0]
    wc = inputs.interface_vectors(int(p.M.sum()), 1, 1, 12)[0]
    # L1 through torch.autograd (DDELMSolveScaled -> ddelm_backward with the scale output)
    sc = torch.tensor(p.scale, dtype=torch.float64, device="cuda", requires_grad=True)
    u = solve_u_scaled(s, f, g, sc)
    ((u - _t(target)[:, None]) ** 2).mean().backward()
    got = [float(sc.grad)]
    # L2 = w . u and L3 = w . c through the binding
    _, _, _, gs2 = s.backward(grad_u=_t(wu), scale=True)
    _, _, _, gs3 = s.backward(grad_c=_t(wc), scale=True)
    got += [gs2, gs3]

    def losses(scale):
        r = odd.solve(dataclasses.replace(p, scale=scale), odd.Options(eps_rel=1e-6))
        ue, ce = r["u_eval"][:, 0], np.concatenate(r["c"])[:, 0]
        return np.array([np.mean((ue - target) ** 2), wu[:, 0] @ ue, wc[:, 0] @ ce])

    def fd4(h):
        Lp2, Lp1, Lm1, Lm2 = (losses(p.scale + j * h) for j in (2, 1, -1, -2))
        return (-Lp2 + 8 * Lp1 - 8 * Lm1 + Lm2) / (12 * h)

    h = 2e-3 * p.scale
    ref_h, ref = fd4(h), fd4(h / 2)
    for k in range(3):
        # halving the step moves the fourth-order difference by about 15x its
        # remaining truncation error; the bound adds that movement to 1e-6
        assert abs(ref_h[k] - ref[k]) <= 1e-5 * abs(ref[k]), (k, ref_h[k], ref[k])
        tol = 1e-6 * abs(ref[k]) + abs(ref_h[k] - ref[k])
        print(f"scale gradient 3x3 {prec} loss {k + 1}: {got[k]:.12e} vs oracle {ref[k]:.12e} "
              f"rel {abs(got[k] - ref[k]) / abs(ref[k]):.2e}")
        assert abs(got[k] - ref[k]) <= tol, (k, got[k], ref[k], tol)
