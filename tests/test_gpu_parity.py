"""GPU path against the FP64 oracle, element by element, through the C ABI."""
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



def _run(D, p, **kw):
    import torch
    s = D.Solver(p, **kw)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    return s, c.cpu().numpy(), mu.cpu().numpy(), u.cpu().numpy(), info, rc


SMALL = [  # nx, ny, M, n_int, e, eps_rel, theta, R, seed
    (2, 2, 12, 40, 3, 1e-6, 0.999, 1, 1),
    (3, 3, 10, 40, 2, 1e-6, 0.5, 2, 2),
    (3, 2, 70, 150, 5, 1e-6, 1.0, 1, 3),      # spans two 64-wide tiles with a ragged tail
    (2, 1, 10, 40, 3, 1e-6, 0.999, 1, 4),     # no cross points: Pi empty
    (4, 3, 20, 60, 3, 1e-6, 0.0, 3, 5),
    (3, 3, 130, 300, 7, 1e-6, 0.999, 1, 6),   # three tiles, ragged
]


@pytest.mark.parametrize("case", SMALL)
def test_assembly_and_local_operators(D, case):
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps, theta=th))
    s = D.Solver(p, theta=th, eps_rel=eps, tol=1e-13, keep_matrices=True)
    for i in range(p.n_sub):
        L = o.loc[i]
        np.testing.assert_allclose(s.inspect(i, 0), L.K, rtol=1e-13, atol=1e-13 * np.abs(L.K).max())
        np.testing.assert_allclose(s.inspect(i, 1), L.Kbar, rtol=1e-13, atol=1e-13 * np.abs(L.Kbar).max())
        np.testing.assert_allclose(s.inspect(i, 2), L.Ahat, rtol=1e-12, atol=1e-13 * np.abs(L.Ahat).max())
        G = slice(L.m - L.nG, L.m)
        Lam = L.Ahat @ L.Kpinv[:, G]                       # -A^i K^+ B^i on Gamma^i
        Psi = (L.K @ L.Kpinv)[G, G]                        # E^T K K^+ E
        Phi = L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:]        # A-bar K-bar^+ E_Delta
        assert close(s.inspect(i, 3), Lam, 1e-9, "s.inspect(i, 3) vs Lam")
        assert close(s.inspect(i, 4), Psi, 1e-9, "s.inspect(i, 4) vs Psi")
        if L.nDl:
            assert close(s.inspect(i, 5), Phi, 1e-9, "s.inspect(i, 5) vs Phi")
    if o.n_pi:
        assert close(s.inspect(0, 6), o.S_Pi, 1e-9, "s.inspect(0, 6) vs o.S_Pi")


@pytest.mark.parametrize("case", SMALL)
def test_solution_matches_oracle(D, case):
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    ref = odd.solve(p, odd.Options(eps_rel=eps, theta=th))
    s, c, mu, u, info, rc = _run(D, p, theta=th, eps_rel=eps, tol=1e-11)
    assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
    n_pi = ref["oracle"].n_pi
    assert close(mu[n_pi:], ref["mu_delta"], 1e-9, "mu[n_pi:] vs ref['mu_delta']")
    if n_pi:
        assert close(mu[:n_pi], ref["mu_pi"], 1e-9, "mu[:n_pi] vs ref['mu_pi']")
    assert close(u, ref["u_eval"], 1e-9, "u vs ref['u_eval']")
    assert info.rel_residual < 1e-10
    assert info.iterations > 0


@pytest.mark.parametrize("eps_rel,tol,pde_err", [(1e-5, 1e-10, 1e-3), (1e-8, 1e-7, 1e-4)])
def test_poisson_2x2_m100_matches_oracle(D, eps_rel, tol, pde_err):
    """2x2, M=100.  The bound is the spread of two backward-stable FP64
    factorisations of the same ridge problem (Householder QR vs SVD): ~3e-11 at
    eps_rel = 1e-5, ~2e-8 at eps_rel = 1e-8."""
    p = inputs.config("poisson_2x2_m100")
    ref = odd.solve(p, odd.Options(eps_rel=eps_rel))
    s, c, mu, u, info, rc = _run(D, p, eps_rel=eps_rel, tol=1e-11)
    assert rc == D.DDELM_OK
    assert close(mu[1:], ref["mu_delta"], tol, "mu[1:] vs ref['mu_delta']")
    assert close(u, ref["u_eval"], tol, "u vs ref['u_eval']")
    assert close(u, p.u_eval_exact, pde_err, "u vs p.u_eval_exact")   # sanity against sin(pi x) sin(pi y)


@pytest.mark.parametrize("case", [SMALL[2], SMALL[5]])
def test_feature_rows_to_rounding(D, case):
    """Every row of K_c and K-bar (tanh point values, fluxes, the change of variables,
    Laplacian rows) within a few units of rounding of the oracle's, relative to
    the row's largest entry: the feature tanh is accurate to ~2e-16 absolute."""
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps, theta=th))
    s = D.Solver(p, theta=th, eps_rel=eps, tol=1e-13, keep_matrices=True)
    worst = 0.0
    for i in range(p.n_sub):
        L = o.loc[i]
        for which, ref in ((0, L.K), (1, L.Kbar), (2, L.Ahat)):
            got = s.inspect(i, which)
            scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
            worst = max(worst, float((np.abs(got - ref) / scale).max()))
    assert worst < 2e-14, worst


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cov,use_Am", [(True, True), (True, False), (False, True), (False, False)])
def test_ablation_variants_match_oracle(D, cov, use_Am, prec):
    """The coarse-space variants of the paper's ablation: K or K_c (change of
    variables, Sec. 3.2) with the plain flux rows A or the modified A_m."""
    p = inputs.small_problem(3, 3, M=24, n_int=70, edge_pts=4, n_rhs=1, seed=19)
    ref = odd.solve(p, odd.Options(eps_rel=1e-6, theta=0.999, use_change_of_vars=cov, use_Am=use_Am))
    s, c, mu, u, info, rc = _run(D, p, theta=0.999, eps_rel=1e-6, tol=1e-12, use_change_of_vars=cov,
                                 use_Am=use_Am, precision=D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED)
    assert rc == D.DDELM_OK
    n_pi = ref["oracle"].n_pi
    assert close(mu[n_pi:], ref["mu_delta"], 1e-9, f"ablation cov={cov} Am={use_Am} {prec} mu")
    assert close(u, ref["u_eval"], 1e-9, f"ablation cov={cov} Am={use_Am} {prec} u")
