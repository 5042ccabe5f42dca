"""Factorisation schemes and the variable-coefficient operator against the FP64
oracle: the FP32-Cholesky scheme (shifted FP32 passes, exact updates, series
polish of the last factor) in both precisions, the CQR2 + series scheme with
FP64 or double-FP32 first factors, the tensor-core tile autotuner, and
-div(a grad u) problems."""
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



def _data(p):
    import torch
    return (torch.tensor(p.f_int, dtype=torch.float64, device="cuda"),
            torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda"))


def _solve(D, p, **kw):
    import torch
    s = D.Solver(p, **kw)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    return s, mu.cpu().numpy(), u.cpu().numpy(), info, rc


SCHEME_CASES = [  # nx, ny, M, n_int, e, eps_rel, R, seed, passes
    (2, 2, 12, 40, 3, 1e-6, 1, 1, 0),
    (3, 3, 130, 300, 7, 1e-6, 2, 6, 0),
    (2, 2, 200, 700, 20, 1e-8, 1, 9, 0),
    (2, 2, 200, 700, 20, 1e-8, 1, 9, 6),
    (3, 2, 90, 260, 9, 1e-7, 1, 4, 0),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", SCHEME_CASES)
def test_fp32_cholesky_scheme(D, case, prec):
    nx, ny, M, nI, e, eps, R, seed, passes = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps))
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    s, mu, u, info, rc = _solve(D, p, eps_rel=eps, tol=1e-11, precision=pr,
                                setup_scheme=D.DDELM_SCHEME_FP32, setup_passes=passes)
    assert rc == D.DDELM_OK
    tol_op = 1e-9 if eps >= 1e-6 else 1e-6
    for i in range(p.n_sub):
        L = o.loc[i]
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], tol_op, "s.inspect(i, 3) vs L.Ahat @ L.Kpinv[:, G]")
        assert close(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G], tol_op, "s.inspect(i, 4) vs (L.K @ L.Kpinv)[G, G]")
        if L.nDl:
            assert close(s.inspect(i, 5), L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:], tol_op, "s.inspect(i, 5) vs L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:]")
    ref = odd.solve(p, odd.Options(eps_rel=eps))
    tol = 1e-8 if eps >= 1e-6 else 1e-7
    assert close(mu[o.n_pi:], ref["mu_delta"], tol, "mu[o.n_pi:] vs ref['mu_delta']")
    assert close(u, ref["u_eval"], tol, "u vs ref['u_eval']")


def test_too_few_fp32_passes_is_reported(D):
    """Two shifted FP32 passes cannot bring a Gram of condition ~1e18 near the identity:
    the setup must fail with a status (the series check or a pivot), never return."""
    p = inputs.small_problem(2, 2, M=200, n_int=700, edge_pts=20, n_rhs=1, seed=9)
    with pytest.raises(D.DDELMError):
        D.Solver(p, eps_rel=1e-8, tol=1e-11, precision=D.DDELM_PREC_MIXED,
                 setup_scheme=D.DDELM_SCHEME_FP32, setup_passes=2)


@pytest.mark.parametrize("scheme", ["fp64 factors", "double-fp32 factors"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", SCHEME_CASES[:3])
def test_cqr2_series_scheme(D, case, prec, scheme):
    """Two Cholesky passes, the third replaced by the series of (I + E)^{-1/2};
    the two factors in FP64 or in double-FP32 arithmetic."""
    nx, ny, M, nI, e, eps, R, seed, _ = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps))
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    s, mu, u, info, rc = _solve(D, p, eps_rel=eps, tol=1e-11, precision=pr,
                                setup_scheme=D.DDELM_SCHEME_CQR2_SERIES if scheme == "fp64 factors"
                                else D.DDELM_SCHEME_CQR2_SERIES_DW)
    assert rc == D.DDELM_OK
    tol_op = 1e-9 if eps >= 1e-6 else 1e-6
    for i in range(p.n_sub):
        L = o.loc[i]
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], tol_op, "s.inspect(i, 3) vs L.Ahat @ L.Kpinv[:, G]")
        assert close(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G], tol_op, "s.inspect(i, 4) vs (L.K @ L.Kpinv)[G, G]")
    ref = odd.solve(p, odd.Options(eps_rel=eps))
    tol = 1e-8 if eps >= 1e-6 else 1e-7
    assert close(mu[o.n_pi:], ref["mu_delta"], tol, "mu[o.n_pi:] vs ref['mu_delta']")
    assert close(u, ref["u_eval"], tol, "u vs ref['u_eval']")


def test_fp32_scheme_uneven(D):
    p = inputs.small_uneven_problem(4, 3, n_rhs=2)
    ref = odd.solve(p, odd.Options(eps_rel=1e-6))
    s, mu, u, info, rc = _solve(D, p, eps_rel=1e-6, tol=1e-11, precision=D.DDELM_PREC_MIXED,
                                setup_scheme=D.DDELM_SCHEME_FP32)
    assert rc == D.DDELM_OK
    n_pi = ref["oracle"].n_pi
    assert close(mu[n_pi:], ref["mu_delta"], 1e-8, "mu[n_pi:] vs ref['mu_delta']")
    assert close(u, ref["u_eval"], 1e-8, "u vs ref['u_eval']")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", [1, 2, 3, 4])
def test_variable_coefficient_operator(D, prec, scheme):
    """-div(a grad u) = f with a = 1 + 0.5 sin(2 pi x) sin(2 pi y): local operators and solution."""
    p = inputs.small_problem(3, 3, M=80, n_int=200, edge_pts=6, n_rhs=2, seed=21, op=inputs.OP_DIFFUSION)
    assert p.op == inputs.OP_DIFFUSION and np.ptp(p.a_int) > 0.5
    o = odd.DDELMOracle(p, odd.Options(eps_rel=1e-6))
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    s, mu, u, info, rc = _solve(D, p, eps_rel=1e-6, tol=1e-11, precision=pr, setup_scheme=scheme,
                                keep_matrices=True)
    assert rc == D.DDELM_OK
    for i in range(p.n_sub):
        L = o.loc[i]
        assert close(s.inspect(i, 0), L.K, 1e-13, "s.inspect(i, 0) vs L.K")  # assembled K_c with the variable-coefficient rows
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], 1e-9, "s.inspect(i, 3) vs L.Ahat @ L.Kpinv[:, G]")
    ref = odd.solve(p, odd.Options(eps_rel=1e-6))
    assert close(mu[o.n_pi:], ref["mu_delta"], 1e-8, "mu[o.n_pi:] vs ref['mu_delta']")
    assert close(u, ref["u_eval"], 1e-8, "u vs ref['u_eval']")


def test_blocked_cholesky_matches_unblocked(D):
    """The blocked FP64 Cholesky (diagonal blocks on the FP64 pipe, panels and
    trailing updates as tensor-core GEMMs) on well-conditioned local problems
    (eps_rel = 1e-4): the same factor and solution as one CTA per matrix."""
    p = inputs.make_problem(2, 2, 300, 1000, 20, scale=32.0, init="paper", seed=5, solutions=[inputs._sin_sin(1, 1)])
    out = {}
    for blocked in (False, True):
        s, mu, u, info, rc = _solve(D, p, eps_rel=1e-4, tol=1e-12, precision=D.DDELM_PREC_MIXED,
                                    setup_scheme=D.DDELM_SCHEME_CQR2_SERIES, chol_blocked=blocked)
        assert rc == D.DDELM_OK
        out[blocked] = (u, s.inspect(0, 10))
        s.close()
    assert close(out[True][0], out[False][0], 1e-11, "blocked Cholesky u")
    assert close(out[True][1], out[False][1], 1e-10, "blocked Cholesky V = R^{-1}")


def test_tile_autotuner(D):
    """The first setup times both tensor-core tile shapes of every phase whose
    products overwrite their output and keeps the faster: the solution is the
    same as with the fixed rule (both shapes are exact slice expansions) and
    the tuner reports what it timed."""
    p = inputs.small_problem(3, 3, M=130, n_int=300, edge_pts=7, n_rhs=1, seed=6)
    ref = odd.solve(p, odd.Options(eps_rel=1e-6))
    sols = {}
    for tune in (False, True):
        s, mu, u, info, rc = _solve(D, p, eps_rel=1e-6, tol=1e-12, precision=D.DDELM_PREC_MIXED, autotune=tune)
        assert rc == D.DDELM_OK
        rep = D.ddelm_inspect(s.h, 0, 11, 4)
        if tune:   # phases timed here or earlier in this process (the choices are cached by shape)
            assert rep[0] > 0 and 0 <= rep[1] <= rep[0] and rep[2] >= 0 and rep[3] <= rep[2] * 1.0001 + 1e-9
        else:
            assert rep[0] == 0
        s.refactor()                                # a second setup with the kept widths
        c2, mu2, u2, info2, rc2 = s.solve(*_data(p))
        assert rc2 == D.DDELM_OK
        sols[tune] = u2.cpu().numpy()
        assert close(u, ref["u_eval"], 1e-9, f"autotune={tune} u")
    assert close(sols[True], sols[False], 1e-10, "autotuned vs rule widths")
