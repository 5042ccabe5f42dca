"""Vanilla DDELM (Sec. 2.2.1, Eq. (schur): no coarse space) on grids with cross
points, on the GPU against the FP64 oracle through the C ABI.  Every cross
point is an interface unknown of its four subdomains (the interface gathers
sum four owners there), with the plain corner flux row.

Tolerance: the spread of two backward-stable FP64 factorisations of the same
ridge problems (Householder QR vs SVD pseudo-inverses in the oracle), measured
on these cases, is at most 2.0e-11 (mu) and 1.7e-10 (u); the bound is 1e-9."""
import numpy as np
import pytest

from oracle import ddelm as odd
from paper_2503_10032_gb300 import inputs
from parity_util import close

pytestmark = pytest.mark.gpu

TOL = 1e-9


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


VAN = [  # nx, ny, M, n_int, e, op, R, seed
    (3, 3, 30, 90, 3, 0, 1, 1),
    (4, 3, 40, 120, 4, 0, 2, 2),
    (3, 3, 70, 160, 5, 0, 1, 3),     # two 64-wide tiles with a ragged tail
    (3, 3, 30, 90, 3, 2, 1, 4),      # biharmonic: two components, four owners at each cross point for both
    (3, 3, 40, 120, 4, 1, 1, 5),     # variable-coefficient diffusion
]


def _problem(case):
    nx, ny, M, nI, e, op, R, seed = case
    return inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed, op=op)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", VAN)
def test_vanilla_solution_matches_oracle(D, case, prec):
    p = _problem(case)
    ref = odd.solve(p, odd.Options(eps_rel=1e-6, theta=0.0, use_coarse=False))
    s, c, mu, u, info, rc = _run(D, p, theta=0.0, eps_rel=1e-6, tol=1e-12, use_coarse=False,
                                 precision=D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED)
    assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
    assert ref["oracle"].n_pi == 0 and mu.shape[0] == ref["oracle"].n_dl
    assert close(mu, ref["mu_delta"], TOL, f"vanilla {case} {prec} mu")
    assert close(u, ref["u_eval"], TOL, f"vanilla {case} {prec} u")
    assert info.rel_residual < 1e-11


@pytest.mark.parametrize("case", [VAN[0], VAN[3]])
def test_vanilla_rows_and_local_operators(D, case):
    """The cross points' Delta rows (point values and the plain corner fluxes)
    and the local operators of every subdomain."""
    p = _problem(case)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=1e-6, theta=0.0, use_coarse=False))
    s = D.Solver(p, theta=0.0, eps_rel=1e-6, tol=1e-13, keep_matrices=True, use_coarse=False)
    for i in range(p.n_sub):
        L = o.loc[i]
        for which, ref in ((0, L.K), (1, L.Kbar), (2, L.Ahat)):
            got = s.inspect(i, which)
            scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
            assert float((np.abs(got - ref) / scale).max()) < 4e-14, (i, which)
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], TOL, f"vanilla {case} Lambda {i}")
        assert close(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G], TOL, f"vanilla {case} Psi {i}")


def test_vanilla_adjoint_matches_oracle(D):
    """dL/d(f, g) through vanilla DDELM against the oracle's linear map."""
    import torch
    p = _problem(VAN[1])
    s, c, mu, u, info, rc = _run(D, p, theta=0.0, eps_rel=1e-6, tol=1e-13, use_coarse=False)
    rng = np.random.default_rng(5)
    wu = rng.standard_normal(u.shape)
    gf, gg, _ = s.backward(grad_u=torch.tensor(wu, device="cuda"))
    q = _problem(VAN[1])
    q.f_int, q.g_bnd = rng.standard_normal(p.f_int.shape), rng.standard_normal(p.g_bnd.shape)
    du = odd.solve(q, odd.Options(eps_rel=1e-6, theta=0.0, use_coarse=False))["u_eval"]
    want = float((wu * du).sum())
    got = float((gf.cpu().numpy() * q.f_int).sum() + (gg.cpu().numpy() * q.g_bnd).sum())
    assert abs(got - want) < TOL * np.linalg.norm(wu) * np.linalg.norm(du), (got, want)


def test_vanilla_needs_theta_zero(D):
    p = _problem(VAN[0])
    with pytest.raises(D.DDELMError) as e:
        D.Solver(p, theta=0.999, use_coarse=False)
    assert e.value.status == D.DDELM_ERR_INVALID_ARG


def test_vanilla_vs_coarse_space_iterations(D):
    """The coarse space's purpose (Sec. 3): on the same problem DDELM-CS needs
    fewer CG iterations than vanilla DDELM, and DDELM-NN fewer still."""
    p = inputs.make_problem(6, 6, 120, 400, 20, scale=12.0, init="paper", seed=31,
                            solutions=[inputs._sin_sin(1, 1)], points="grid")
    its = {}
    for name, kw in (("ddelm", dict(theta=0.0, use_coarse=False)), ("cs", dict(theta=0.0)),
                     ("nn", dict(theta=0.999))):
        s, c, mu, u, info, rc = _run(D, p, eps_rel=1e-8, tol=1e-9, max_iters=20000, **kw)
        assert rc == D.DDELM_OK
        its[name] = info.iterations
    print("CG iterations on a 6x6 grid:", its)
    assert its["nn"] < its["cs"] < its["ddelm"]
