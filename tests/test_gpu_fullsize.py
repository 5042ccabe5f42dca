"""Full-size workloads, in the launch configuration bench.py times (theta 0.999,
eps_rel 1e-8, CG to relative residual 1e-8), against the oracle on what it can
compute at that size: its stored full solution of the 8x8, M=400 workload
(tests/golden, written by make_fullsize_golden.py), the local operators of
sampled subdomains of every workload, and properties that hold at any size
(true residual, manufactured-solution error, CUDA-graph replay)."""
import os

import numpy as np
import pytest

from oracle import ddelm as odd
from paper_2503_10032_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BENCH = dict(theta=0.999, eps_rel=1e-8, tol=1e-8, max_iters=20000)


@pytest.fixture(scope="module")
def D():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_10032_gb300 import build
    build.build()
    from paper_2503_10032_gb300 import ddelm
    return ddelm


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _solve(D, p, **kw):
    import torch
    s = D.Solver(p, **kw)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    return s, c.cpu().numpy(), mu.cpu().numpy(), u.cpu().numpy(), info, rc


def _local_parity(D, s, p, subs, tol):
    o = odd.DDELMOracle(p, odd.Options(eps_rel=BENCH["eps_rel"], theta=BENCH["theta"]), only=list(subs))
    for i in subs:
        L = o.loc[i]
        G = slice(L.m - L.nG, L.m)
        assert _rel(s.inspect(i, 3), L.Ahat @ L.Kpinv[:, G]) < tol, i
        assert _rel(s.inspect(i, 4), (L.K @ L.Kpinv)[G, G]) < tol, i
        if L.nDl:
            assert _rel(s.inspect(i, 5), L.Abar @ L.Kbar_pinv[:, L.m - L.nDl:]) < tol, i


def _free(s):
    import torch
    s.close()
    del s
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_poisson_8x8_m400_against_stored_oracle_solution(D, prec):
    p = inputs.config("poisson_8x8_m400")
    mu_ref = np.loadtxt(os.path.join(GOLDEN, "poisson_8x8_m400_mu_delta.txt")).reshape(-1, 1)
    u_ref = np.loadtxt(os.path.join(GOLDEN, "poisson_8x8_m400_u_eval.txt")).reshape(-1, 1)
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    s, c, mu, u, info, rc = _solve(D, p, precision=pr, **BENCH)
    assert rc == D.DDELM_OK and info.rel_residual < 1e-8
    n_pi = s.sizes.n_pi
    # stopping at residual 1e-8 leaves a CG error of order cond * 1e-8 in mu;
    # u (the method's output) is closer
    assert _rel(mu[n_pi:], mu_ref) < 1e-6
    assert _rel(u, u_ref) < 1e-7
    x_e = p.x_eval
    u_exact = np.sin(2 * np.pi * x_e[:, 0]) * np.cos(3 * np.pi * x_e[:, 1])
    assert _rel(u[:, 0], u_exact) < 1e-3
    _local_parity(D, s, p, [0, 27, 63], 1e-6)
    _free(s)
    # to a tight residual the GPU solution meets the oracle's
    s, c, mu, u, info, rc = _solve(D, p, precision=pr, **dict(BENCH, tol=1e-11))
    assert rc == D.DDELM_OK
    assert _rel(mu[n_pi:], mu_ref) < 1e-7
    assert _rel(u, u_ref) < 1e-7
    _free(s)


def test_poisson_16x16_uneven(D):
    p = inputs.config("poisson_16x16_uneven")
    s, c, mu, u, info, rc = _solve(D, p, precision=D.DDELM_PREC_MIXED, **BENCH)
    assert rc == D.DDELM_OK and info.rel_residual < 1e-8
    x_e = p.x_eval
    u_exact = np.sin(np.pi * x_e[:, 0]) * np.sin(np.pi * x_e[:, 1])
    assert _rel(u[:, 0], u_exact) < 1e-3
    # smallest, largest and a middle subdomain
    order = np.argsort(p.M)
    _local_parity(D, s, p, [int(order[0]), int(order[-1]), 136], 1e-6)
    _free(s)


def test_diffusion_32x32_m1000_16_rhs(D):
    p = inputs.config("diffusion_32x32_m1000_r16")
    s, c, mu, u, info, rc = _solve(D, p, precision=D.DDELM_PREC_MIXED, **BENCH)
    assert rc == D.DDELM_OK and info.rel_residual < 1e-8
    assert u.shape[1] == 16
    x_e = p.x_eval
    k = 0
    for a in range(1, 5):
        for b in range(1, 5):
            u_exact = np.sin(a * np.pi * x_e[:, 0]) * np.sin(b * np.pi * x_e[:, 1])
            assert _rel(u[:, k], u_exact) < 1e-3, (a, b)
            k += 1
    _local_parity(D, s, p, [0, 529], 1e-6)
    _free(s)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_is_bitwise_identical(D, prec):
    """Setup and solve replayed from captured CUDA graphs give the same bits as direct launches."""
    import torch
    p = inputs.small_uneven_problem(4, 3, n_rhs=2, seed=5)
    pr = D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    outs = {}
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s = D.Solver(p, eps_rel=1e-6, tol=1e-11, precision=pr, graphs=graphs, stream=stream)
            res = []
            for _ in range(3):
                s.refactor()
                c, mu, u, info, rc = s.solve(f, g)
                assert rc == D.DDELM_OK
                res.append(mu.cpu().numpy())
        torch.cuda.synchronize()
        assert all(np.array_equal(res[0], r) for r in res[1:])
        plan = D.ddelm_inspect(s.h, 0, 9, 6)
        assert (plan[4], plan[5]) == ((1.0, 1.0) if graphs else (0.0, 0.0))
        outs[graphs] = res[0]
        s.close()
    assert np.array_equal(outs[False], outs[True])
