"""The no-allocation entry point against the regular path (GPU).

ddelm_local_lstsq_static serves callers that cannot allocate device memory
(its scratch is a static device array).  On a single subdomain the interface
is empty, so ddelm_solve returns c = K^+ f for the same K; the static entry
point, given that K (from ddelm_inspect) and f, must return the same c, on two
calls in a row (the array keeps the previous call's contents).
"""
import numpy as np
import pytest

from paper_2503_10032_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_static_scratch_lstsq_matches_solve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_10032_gb300 import build
    build.build()
    from paper_2503_10032_gb300 import ddelm as D
    p = inputs.make_problem(1, 1, 100, 400, 20, scale=2.0, init="uniform", seed=31,
                            solutions=[inputs._sin_sin(1, 1), inputs._sin2pix_cos3piy()], name="one")
    eps = 1e-6
    s = D.Solver(p, eps_rel=eps, tol=1e-11, keep_matrices=True)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c_ref, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    assert rc == D.DDELM_OK and s.sizes.n_delta == 0
    K = s.inspect(0, 0)
    m, M = K.shape
    F = np.vstack([p.f_int, p.g_bnd])          # local rows: interior, then boundary (no interface)
    assert F.shape[0] == m
    dK = torch.tensor(K, device="cuda")
    dF = torch.tensor(F, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ref = c_ref.cpu().numpy()
    for _ in range(2):
        dC = torch.full((M, F.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
        rc = D.ddelm_local_lstsq_static(dK.data_ptr(), m, M, dF.data_ptr(), F.shape[1], eps, dC.data_ptr(), stream)
        assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
        c = dC.cpu().numpy()
        assert np.linalg.norm(c - ref) / np.linalg.norm(ref) < 1e-9
    # sizes beyond the static maximum are rejected, not run
    rc = D.ddelm_local_lstsq_static(dK.data_ptr(), 100000, M, dF.data_ptr(), 1, eps, dC.data_ptr(), stream)
    assert rc == D.DDELM_ERR_INVALID_ARG
