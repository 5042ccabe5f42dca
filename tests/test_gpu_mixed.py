"""Mixed precision: every setup GEMM on the tensor cores (BF16 slices, FP32
TMEM accumulation, FP64 combination) against the FP64 oracle."""
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



CASES = [  # nx, ny, M, n_int, e, eps_rel, theta, R, seed
    (2, 2, 12, 40, 3, 1e-6, 0.999, 1, 1),
    (3, 2, 70, 150, 5, 1e-6, 1.0, 1, 3),
    (3, 3, 130, 300, 7, 1e-6, 0.999, 2, 6),
    (2, 2, 200, 700, 20, 1e-8, 0.999, 1, 9),
]


@pytest.mark.parametrize("case", CASES)
def test_mixed_local_operators_and_solution(D, case):
    import torch
    nx, ny, M, nI, e, eps, th, R, seed = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=R, seed=seed)
    o = odd.DDELMOracle(p, odd.Options(eps_rel=eps, theta=th))
    s = D.Solver(p, theta=th, eps_rel=eps, tol=1e-11, precision=D.DDELM_PREC_MIXED)
    tol_op = 1e-9 if eps >= 1e-6 else 1e-6
    for i in range(p.n_sub):
        L = o.loc[i]
        G = slice(L.m - L.nG, L.m)
        assert close(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G], tol_op, "s.inspect(i, 3) vs L.Ahat @ L.Kpinv[:, G]")
        assert close(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G], tol_op, "s.inspect(i, 4) vs (L.K @ L.Kpinv)[G, G]")
        if L.nDl:
            assert close(s.inspect(i, 5), L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:], tol_op, "s.inspect(i, 5) vs L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:]")
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    ref = odd.solve(p, odd.Options(eps_rel=eps, theta=th))
    tol = 1e-8 if eps >= 1e-6 else 1e-7
    assert rc == D.DDELM_OK
    assert close(mu.cpu().numpy()[o.n_pi:], ref["mu_delta"], tol, "mu.cpu().numpy()[o.n_pi:] vs ref['mu_delta']")
    assert close(u.cpu().numpy(), ref["u_eval"], tol, "u.cpu().numpy() vs ref['u_eval']")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_subdomains(D, prec):
    """Per-subdomain neuron counts, collocation counts and edge point counts all differ."""
    import torch
    p = inputs.small_uneven_problem(4, 3, n_rhs=2)
    assert len(set(p.M.tolist())) > 3 and len(set(p.edge_pts.tolist())) > 2
    ref = odd.solve(p, odd.Options(eps_rel=1e-6))
    s = D.Solver(p, eps_rel=1e-6, tol=1e-11,
                 precision=D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    assert rc == D.DDELM_OK
    n_pi = ref["oracle"].n_pi
    assert close(mu.cpu().numpy()[n_pi:], ref["mu_delta"], 1e-8, "mu.cpu().numpy()[n_pi:] vs ref['mu_delta']")
    assert close(u.cpu().numpy(), ref["u_eval"], 1e-8, "u.cpu().numpy() vs ref['u_eval']")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_setup_waves_give_identical_results(D, prec):
    """Subdomains set up in waves that share scratch slots give the same bits."""
    import torch
    p = inputs.small_uneven_problem(4, 3, n_rhs=1, seed=17)
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    outs = []
    for wave in (0, 5, 1):
        s = D.Solver(p, eps_rel=1e-6, tol=1e-11, precision=pr, setup_wave=wave)
        c, mu, u, info, rc = s.solve(f, g)
        torch.cuda.synchronize()
        assert rc == D.DDELM_OK
        outs.append(mu.cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
