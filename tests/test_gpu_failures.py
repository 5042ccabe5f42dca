"""Failure detection through the C ABI (GPU): every failure is made on the host
(an iteration cap, a NaN in the data, a neuron whose features vanish, a grid
barrier told to wait for one arrival more than the grid has) and must come back
as a status, with the CUDA context still usable afterwards."""
import numpy as np
import pytest

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


def _prec(D, prec):
    return D.DDELM_PREC_FP64 if prec == "fp64" else D.DDELM_PREC_MIXED


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_cap_reports_not_converged(D, prec):
    p = inputs.small_problem(3, 3, M=30, n_int=90, edge_pts=4, seed=3)
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12, max_iters=1, max_refine=1, precision=_prec(D, prec))
    c, mu, u, info, rc = s.solve(_t(p.f_int), _t(p.g_bnd))
    assert rc == D.DDELM_ERR_NOT_CONVERGED
    assert info.iterations >= 1 and info.rel_residual > 1e-12
    assert np.all(np.isfinite(c.cpu().numpy())) and np.all(np.isfinite(u.cpu().numpy()))   # outputs written


@pytest.mark.parametrize("where", ["f", "g"])
def test_nan_in_data_is_not_silent(D, where):
    p = inputs.small_problem(3, 3, M=30, n_int=90, edge_pts=4, seed=3)
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12)
    f, g = p.f_int.copy(), p.g_bnd.copy()
    (f if where == "f" else g)[5, 0] = np.nan
    c, mu, u, info, rc = s.solve(_t(f), _t(g))
    assert rc == D.DDELM_ERR_NOT_CONVERGED
    assert np.isnan(info.rel_residual)
    # the handle still solves clean data
    c, mu, u, info, rc = s.solve(_t(p.f_int), _t(p.g_bnd))
    assert rc == D.DDELM_OK and info.rel_residual < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vanishing_neuron_is_rank_deficient(D, prec):
    """w_hat = b_hat = 0 makes a neuron's features vanish everywhere (tanh 0 = 0), a
    zero column of K_c^i and K-bar^i: without the ridge (eps_rel = 0, the
    Moore-Penrose reading) the factorisation meets a zero pivot and reports the
    subdomain; with the ridge the same problem sets up."""
    import torch
    p = inputs.small_problem(3, 3, M=30, n_int=90, edge_pts=4, seed=3)
    sub = 4
    j = int(p.M[:sub].sum()) + 7
    p.w_hat[j] = 0.0
    p.b_hat[j] = 0.0
    pa = D.ProblemArgs(p, D.make_options(eps_rel=0.0, precision=_prec(D, prec)))
    sz = D.ddelm_query(pa)
    ws = torch.empty(int(sz.workspace_bytes) + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    rc, h, info_sub = D.ddelm_setup(pa, ptr, int(sz.workspace_bytes), torch.cuda.current_stream().cuda_stream)
    assert rc == D.DDELM_ERR_RANK_DEFICIENT and info_sub == sub
    if h.value:
        D.ddelm_destroy(h)
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12, precision=_prec(D, prec))
    c, mu, u, info, rc = s.solve(_t(p.f_int), _t(p.g_bnd))
    assert rc == D.DDELM_OK


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stalled_barrier_times_out_and_context_survives(D, prec):
    """Every grid barrier of the interface solve waits for an arrival that never
    comes; after its 20 ms limit it sets the error word, every CTA returns, and
    the call reports DDELM_ERR_TIMEOUT.  The same process then solves normally."""
    import time
    p = inputs.small_problem(3, 3, M=30, n_int=90, edge_pts=4, seed=3)
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12, precision=_prec(D, prec), barrier_timeout_ms=20,
                 inject_barrier_stall=True, graphs=False)
    t0 = time.time()
    with pytest.raises(D.DDELMError) as e:
        s.solve(_t(p.f_int), _t(p.g_bnd))
    assert e.value.status == D.DDELM_ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    s.close()
    s = D.Solver(p, eps_rel=1e-6, tol=1e-12, precision=_prec(D, prec))
    c, mu, u, info, rc = s.solve(_t(p.f_int), _t(p.g_bnd))
    assert rc == D.DDELM_OK and info.rel_residual < 1e-12
