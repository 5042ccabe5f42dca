"""Adjoint (ddelm_backward) against the forward solve, the oracle and finite
differences; gradients of a solution loss w.r.t. Fourier forcing coefficients."""
import numpy as np
import pytest

from oracle import ddelm as odd
from paper_2503_10032_gb300 import inputs

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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


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
    assert _rel(g_gpu, g_ref) < (1e-6 if prec == "fp64" else 1e-5)


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
    assert _rel(grad, fd) < 1e-6
    # oracle: u is linear in a; du/da_pq = solve(basis column pq, g = 0)
    q = inputs.make_problem(3, 3, 40, 120, 4, scale=8.0, init="paper", seed=41,
                            solutions=[inputs.fourier_forcing(a0)], n_eval=16)
    q.f_int = basis
    q.g_bnd = np.zeros((p.g_bnd.shape[0], 16))
    ref = odd.solve(q, odd.Options(eps_rel=1e-6))
    U = ref["u_eval"]                          # [n_eval, 16]
    u_now = U @ a0
    grad_ref = 2.0 / len(u_now) * U.T @ (u_now - np.sin(np.pi * p.x_eval[:, 0]) * np.sin(np.pi * p.x_eval[:, 1]))
    assert _rel(grad, grad_ref) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_scale_gradient(D, prec):
    """dL/ds for the hidden-layer scale s (w = s w_hat, b = s b_hat), with
    L = mean (u - sin(pi x) sin(pi y))^2: the tangent path against central
    differences of the FP64 oracle's solution."""
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
    ut = _t(target)[:, None]
    sc = torch.tensor(p.scale, dtype=torch.float64, device="cuda", requires_grad=True)
    u = solve_u_scaled(s, f, g, sc)
    L = ((u - ut) ** 2).mean()
    L.backward()
    grad = float(sc.grad)

    def loss_oracle(scale):
        q = dataclasses.replace(p, scale=scale)
        uo = odd.solve(q, odd.Options(eps_rel=1e-6))["u_eval"][:, 0]
        return float(np.mean((uo - target) ** 2))

    h = 1e-4 * p.scale
    fd = (loss_oracle(p.scale + h) - loss_oracle(p.scale - h)) / (2 * h)
    assert abs(grad - fd) <= 1e-5 * abs(fd), (grad, fd)
    # the tangent of u itself against the oracle's central difference
    from paper_2503_10032_gb300.tangent import scale_tangent
    _, du = scale_tangent(s, f, g)
    up = odd.solve(dataclasses.replace(p, scale=p.scale + h), odd.Options(eps_rel=1e-6))["u_eval"]
    um = odd.solve(dataclasses.replace(p, scale=p.scale - h), odd.Options(eps_rel=1e-6))["u_eval"]
    assert _rel(du.cpu().numpy(), (up - um) / (2 * h)) < 1e-5
