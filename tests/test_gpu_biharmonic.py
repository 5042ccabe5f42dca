"""Biharmonic operator (the coupled system of Sec. 2.1) on the GPU against the
FP64 oracle, through the C ABI: fourth-order interior rows, two boundary and
two interface components per point, the per-component change of variables
and A_m rows, the reweighted system (derivatives of order k times H^k), the solution in
both precisions.

Tolerances: the spread of two backward-stable FP64 factorisations of the same
ridge problems (oracle with Householder-QR vs SVD pseudo-inverses), measured
on these cases, is at most 5.8e-11 (mu) and 1.8e-9 (u, the 3x3 two-RHS
case); the bounds below are 1e-9 (mu) and 5e-9 (u)."""
import numpy as np
import pytest

from oracle import ddelm as odd
from paper_2503_10032_gb300 import inputs
from parity_util import close

pytestmark = pytest.mark.gpu

TOL_MU, TOL_U = 1e-9, 5e-9


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_10032_gb300 import build
    build.build()
    from paper_2503_10032_gb300 import ddelm
    return ddelm


def _run(D, p, **kw):
    import torch
    s = D.Solver(p, **kw)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    return s, c.cpu().numpy(), mu.cpu().numpy(), u.cpu().numpy(), info, rc


BIH = [  # nx, ny, M, n_int, e, eps_rel, theta, R, seed
    (2, 2, 20, 60, 3, 1e-6, 0.999, 1, 1),
    (3, 3, 40, 120, 4, 1e-6, 0.999, 2, 2),
    (3, 2, 70, 160, 5, 1e-6, 1.0, 1, 3),      # two 64-wide tiles with a ragged tail
    (2, 1, 20, 60, 3, 1e-6, 0.999, 1, 4),     # no cross points: Pi empty
    (3, 3, 40, 120, 3, 1e-6, 0.0, 1, 5),
    (3, 3, 130, 300, 6, 1e-6, 0.999, 1, 6),   # three tiles, ragged
]


def _problem(case):
    nx, ny, M, nI, e, eps, th, R, seed = case
    return inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed, op=inputs.OP_BIHARMONIC)


@pytest.mark.parametrize("case", [BIH[1], BIH[2], BIH[5]])
def test_biharmonic_rows_to_rounding(D, case):
    """Every row of K_c, K-bar and A_m (H^4 Lap^2 phi, phi and H^2 Lap phi at
    boundary and interface points, both weighted fluxes, both components'
    change of variables and corner rows) within a few units of rounding of the
    oracle's, relative to the row's largest entry."""
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = _problem(case)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps, theta=th))
    s = D.Solver(p, theta=th, eps_rel=eps, tol=1e-13, keep_matrices=True)
    worst = 0.0
    for i in range(p.n_sub):
        L = o.loc[i]
        for which, ref in ((0, L.K), (1, L.Kbar), (2, L.Ahat)):
            got = s.inspect(i, which)
            assert got.shape == ref.shape
            scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
            worst = max(worst, float((np.abs(got - ref) / scale).max()))
    assert worst < 4e-14, worst


@pytest.mark.parametrize("case", BIH)
def test_biharmonic_local_operators(D, case):
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = _problem(case)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps, theta=th))
    s = D.Solver(p, theta=th, eps_rel=eps, tol=1e-13, keep_matrices=True)
    for i in range(p.n_sub):
        L = o.loc[i]
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], 1e-9, f"biharmonic {case} Lambda {i}")
        assert close(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G], 1e-9, f"biharmonic {case} Psi {i}")
        if L.nDl:
            assert close(s.inspect(i, 5), L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:], 1e-9, f"biharmonic {case} Phi {i}")
    if o.n_pi:
        assert close(s.inspect(0, 6), o.S_Pi, 1e-9, f"biharmonic {case} S_Pi")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", BIH)
def test_biharmonic_solution_matches_oracle(D, case, prec):
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = _problem(case)
    ref = odd.solve(p, odd.Options(eps_rel=eps, theta=th))
    s, c, mu, u, info, rc = _run(D, p, theta=th, eps_rel=eps, tol=1e-12,
                                 precision=D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED)
    assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
    n_pi = ref["oracle"].n_pi
    assert mu.shape[0] == n_pi + ref["oracle"].n_dl
    assert close(mu[n_pi:], ref["mu_delta"], TOL_MU, f"biharmonic {case} {prec} mu_Delta")
    if n_pi:
        assert close(mu[:n_pi], ref["mu_pi"], TOL_MU, f"biharmonic {case} {prec} mu_Pi")
    assert close(u, ref["u_eval"], TOL_U, f"biharmonic {case} {prec} u")
    assert info.rel_residual < 1e-11


@pytest.mark.parametrize("use_Am", [True, False])
def test_biharmonic_flux_variants(D, use_Am):
    """A_m and the plain flux rows A for both components."""
    p = _problem(BIH[1])
    ref = odd.solve(p, odd.Options(eps_rel=1e-6, theta=0.999, use_Am=use_Am))
    s, c, mu, u, info, rc = _run(D, p, theta=0.999, eps_rel=1e-6, tol=1e-12, use_Am=use_Am)
    assert rc == D.DDELM_OK
    n_pi = ref["oracle"].n_pi
    assert close(mu[n_pi:], ref["mu_delta"], TOL_MU, f"biharmonic Am={use_Am} mu")
    assert close(u, ref["u_eval"], TOL_U, f"biharmonic Am={use_Am} u")


def test_biharmonic_adjoint_matches_oracle_jacobian(D):
    """dL/d(f, g) of a linear loss through the biharmonic solve (reweighted data)
    against the oracle: u is linear in (f, g), so the oracle's u for two
    perturbed data sets fixes the directional derivatives exactly."""
    import torch
    p = _problem(BIH[1])
    s, c, mu, u, info, rc = _run(D, p, theta=0.999, eps_rel=1e-6, tol=1e-13)
    rng = np.random.default_rng(3)
    wu = rng.standard_normal(u.shape)
    gf, gg, _ = s.backward(grad_u=torch.tensor(wu, device="cuda"))
    df, dg = rng.standard_normal(p.f_int.shape), rng.standard_normal(p.g_bnd.shape)
    q = inputs.small_problem(3, 3, M=40, n_int=120, edge_pts=4, n_rhs=2, seed=2, op=inputs.OP_BIHARMONIC)
    q.f_int, q.g_bnd = df, dg
    du = odd.solve(q, odd.Options(eps_rel=1e-6, theta=0.999))["u_eval"]   # u(df, dg): the map is linear
    want = float((wu * du).sum())
    got = float((gf.cpu().numpy() * df).sum() + (gg.cpu().numpy() * dg).sum())
    # the map's relative parity (<= 5e-9, module docstring) bounds the error by |w| |du|
    assert abs(got - want) < 5e-9 * np.linalg.norm(wu) * np.linalg.norm(du), (got, want)


def test_biharmonic_manufactured_solution(D):
    """Lap^2 u = 4 pi^4 u with u = sin(pi x) sin(pi y), u and Lap u on the
    boundary: the GPU solution on a 2x2 grid with 150 neurons per subdomain."""
    p = inputs.make_problem(2, 2, 150, 400, 14, scale=4.0, init="paper", seed=11,
                            solutions=[inputs._sin_sin(1, 1)], op=inputs.OP_BIHARMONIC, points="grid")
    s, c, mu, u, info, rc = _run(D, p, eps_rel=1e-8, tol=1e-10)
    assert rc == D.DDELM_OK
    assert close(u, p.u_eval_exact, 1e-3, "biharmonic manufactured u")


def test_biharmonic_scale_gradient_unsupported(D):
    import torch
    p = _problem(BIH[0])
    s, c, mu, u, info, rc = _run(D, p, eps_rel=1e-6, tol=1e-12)
    gu = torch.ones(u.shape, dtype=torch.float64, device="cuda")
    rc, _, _ = D.ddelm_backward(s.h, 0, gu.data_ptr(), 0, 0, torch.cuda.current_stream().cuda_stream,
                                want_scale=True)
    assert rc == D.DDELM_ERR_UNSUPPORTED
