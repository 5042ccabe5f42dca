"""The no-allocation entry point ddelm_local_lstsq_static (GPU).

It serves callers that cannot allocate device memory (code running where
cudaMalloc is not allowed, or that is handed only fixed buffers): its scratch is
a static device array.  Its result C = K^+ F for one local ELM matrix is checked
against the FP64 oracle's ridge pseudo-inverse (Householder QR of [K; eps I],
numpy/LAPACK), on two calls in a row each time (the array keeps the previous
call's contents), at a regular size, at the limits M = 256, R = 16, and with a
single neuron on a very tall matrix; a rank-deficient K without ridge must be
reported, and sizes beyond the array rejected with a reason.  This file runs
last (pytest collects it last), so a failure here leaves every other test run.
"""
import numpy as np
import pytest

from oracle import ddelm as odd
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


def _local_matrix(M, n_int, n_bnd, R, seed, scale=2.0):
    """One subdomain's ELM rows on [0, 1]^2: -Laplacian of tanh features at
    interior points, point values at boundary points (seeded), and data F."""
    rng = np.random.default_rng(seed)
    w = scale * rng.uniform(-1, 1, (M, 2))
    b = scale * rng.uniform(-1, 1, M)
    xi = rng.uniform(0, 1, (n_int, 2))
    t = rng.uniform(0, 1, n_bnd)
    xb = np.stack([t, (np.arange(n_bnd) % 2).astype(float)], 1)
    K = np.vstack([odd.L_phi(w, b, xi, 0), odd.phi(w, b, xb)])
    F = rng.standard_normal((K.shape[0], R))
    return K, F


def _static(D, K, F, eps):
    import torch
    m, M = K.shape
    R = F.shape[1]
    dK = torch.tensor(K, dtype=torch.float64, device="cuda")
    dF = torch.tensor(F, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):   # two calls in a row on the shared array
        dC = torch.full((M, R), float("nan"), dtype=torch.float64, device="cuda")
        rc = D.ddelm_local_lstsq_static(dK.data_ptr(), m, M, dF.data_ptr(), R, eps, dC.data_ptr(), stream)
        outs.append((rc, dC.cpu().numpy()))
    return outs


def _oracle(K, F, eps):
    pinv, _ = odd._ridge_pinv(K, eps)
    return pinv @ F


@pytest.mark.parametrize("M,n_int,n_bnd,R,eps,tol", [
    (100, 400, 84, 2, 1e-4, 1e-10),     # regular size, moderate ridge
    (100, 400, 84, 2, 1e-6, 1e-8),
    (256, 700, 164, 16, 1e-4, 1e-10),   # the limits M = 256, R = 16 (fits the array)
])
def test_static_matches_oracle_ridge_solve(D, M, n_int, n_bnd, R, eps, tol):
    K, F = _local_matrix(M, n_int, n_bnd, R, seed=31 + M)
    ref = _oracle(K, F, eps)
    for rc, C in _static(D, K, F, eps):
        assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
        assert close(C, ref, tol, f"static lstsq M={M} R={R} eps={eps}")


def test_static_single_neuron_tall(D):
    """M = 1 on 300000 rows: C = K^T F / (K^T K + eps^2), eps^2 = eps_rel^2 |K|^2."""
    rng = np.random.default_rng(5)
    K = rng.standard_normal((300000, 1))
    F = 3.0 * K + rng.standard_normal((300000, 1))
    eps = 1e-3
    ref = _oracle(K, F, eps)
    nk2 = float((K * K).sum())
    closed = (K * F).sum() / (nk2 + eps * eps * nk2)
    assert abs(ref[0, 0] - closed) <= 1e-12 * abs(closed)
    for rc, C in _static(D, K, F, eps):
        assert rc == D.DDELM_OK, D.ddelm_status_string(rc)
        assert abs(C[0, 0] - closed) <= 1e-12 * abs(closed)


def test_static_rank_deficient_and_oversize(D):
    import torch
    K, F = _local_matrix(60, 200, 40, 1, seed=77)
    K[:, 0] = 0.0                       # a neuron whose features all vanish
    for rc, C in _static(D, K, F, 0.0):   # Moore-Penrose reading: the factorisation must fail
        assert rc == D.DDELM_ERR_RANK_DEFICIENT, D.ddelm_status_string(rc)
    for rc, C in _static(D, K, F, 1e-4):  # with the ridge the same K is solvable
        assert rc == D.DDELM_OK
        assert close(C, _oracle(K, F, 1e-4), 1e-10, "static lstsq ridge on a zero column")
    # sizes beyond the static maximum are rejected, not run, with the reason
    dK = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    rc = D.ddelm_local_lstsq_static(dK.data_ptr(), 100000, 100, dK.data_ptr(), 1, 1e-6, dK.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == D.DDELM_ERR_INVALID_ARG
    assert "static array" in D._lib.ddelm_last_error().decode()
