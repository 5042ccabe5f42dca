"""The two tensor-core tile shapes of the MIXED setup: the level-group shape
(128 x 64 tiles, four slice levels per accumulator group, or 128 x 128 with two)
and the all-levels shape (128 x 48 tiles, every level of a 32-wide k block in one
shared-memory stage).  Both compute the same integer level sums of the same
slices and combine them exactly, so where the level-group rule takes the
four-level integer combination (every contraction of at most 1024) the local
operators of the two agree bit for bit; with longer contractions (two k-chunks
in the all-levels shape, the FP64 level combination in the 128-wide one) they
agree to rounding, and both match the FP64 oracle."""
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


def _setup_and_solve(D, p, **kw):
    import torch
    s = D.Solver(p, **kw)
    f = torch.tensor(p.f_int, dtype=torch.float64, device="cuda")
    g = torch.tensor(p.g_bnd, dtype=torch.float64, device="cuda")
    c, mu, u, info, rc = s.solve(f, g)
    torch.cuda.synchronize()
    assert rc == D.DDELM_OK
    return s, mu.cpu().numpy(), u.cpu().numpy()


def _operators(D, s, subs):
    """Lambda, Psi, Phi and V of the given subdomains."""
    out = []
    for i in subs:
        m, M, nG, nDl = (int(v) for v in D.ddelm_inspect(s.h, i, 7, 4))
        out.append(D.ddelm_inspect(s.h, i, 3, nG * nG))
        out.append(D.ddelm_inspect(s.h, i, 4, nG * nG))
        if nDl > 0:
            out.append(D.ddelm_inspect(s.h, i, 5, nDl * nDl))
        out.append(D.ddelm_inspect(s.h, i, 10, M * M))
    return out


SHORT_K = [  # nx, ny, M, n_int, edge points, eps_rel, seed: every contraction <= 1024
    (3, 3, 130, 300, 7, 1e-6, 6),
    (2, 2, 200, 700, 20, 1e-8, 9),
    (3, 2, 90, 260, 9, 1e-7, 4),
]


@pytest.mark.parametrize("case", SHORT_K)
def test_all_levels_bitwise_equal_to_level_groups(D, case):
    nx, ny, M, nI, e, eps, seed = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=1, seed=seed)
    kw = dict(eps_rel=eps, tol=1e-11, precision=D.DDELM_PREC_MIXED, autotune=False)
    s1, mu1, u1 = _setup_and_solve(D, p, tc_tiles=1, **kw)
    s2, mu2, u2 = _setup_and_solve(D, p, tc_tiles=2, **kw)
    subs = sorted({0, nx * ny // 2, nx * ny - 1})
    for a, b in zip(_operators(D, s1, subs), _operators(D, s2, subs)):
        assert a.shape == b.shape
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    assert np.array_equal(u1, u2) and np.array_equal(mu1, mu2)
    ref = odd.solve(p, odd.Options(eps_rel=eps))
    # the oracle spread of the ridge problems grows as eps_rel falls (the same
    # bounds as the factorisation-scheme tests)
    assert close(u2, ref["u_eval"], 1e-8 if eps >= 1e-6 else 1e-7, "all-levels u")


def test_all_levels_two_k_chunks(D):
    """m > 1024 interior and boundary rows: the Grams' contractions take two
    k-chunks.  The all-levels shape and the 128 x 64 level-group shape (both
    exact integer level sums over the chunks) agree bit for bit; the 128 x 128
    shape's FP64 level combination rounds, so it is checked against the
    oracle only (its operators differ from the exact ones by ~1e-10, the
    rounding amplified by the ridge factorisations)."""
    p = inputs.small_problem(2, 2, M=160, n_int=1150, edge_pts=16, n_rhs=1, seed=12)
    eps = 1e-7
    kw = dict(eps_rel=eps, tol=1e-11, precision=D.DDELM_PREC_MIXED, autotune=False)
    s3, mu3, u3 = _setup_and_solve(D, p, tc_tiles=3, **kw)
    s2, mu2, u2 = _setup_and_solve(D, p, tc_tiles=2, **kw)
    s1, mu1, u1 = _setup_and_solve(D, p, tc_tiles=1, **kw)
    m = int(D.ddelm_inspect(s2.h, 0, 7, 4)[0])
    assert m > 1024
    for a, b in zip(_operators(D, s3, [0, 3]), _operators(D, s2, [0, 3])):
        assert a.shape == b.shape
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    assert np.array_equal(u3, u2)
    ref = odd.solve(p, odd.Options(eps_rel=eps))
    assert close(u2, ref["u_eval"], 1e-8, "all-levels u, two k-chunks")
    assert close(u1, ref["u_eval"], 1e-8, "128-wide level-group u")


def test_all_levels_degenerate_sizes(D):
    """Tiny subdomains: products narrower than one 48-wide tile, contractions
    shorter than one k block."""
    p = inputs.small_problem(2, 2, M=12, n_int=40, edge_pts=3, n_rhs=2, seed=1)
    kw = dict(eps_rel=1e-6, tol=1e-12, precision=D.DDELM_PREC_MIXED, autotune=False)
    s2, mu2, u2 = _setup_and_solve(D, p, tc_tiles=2, **kw)
    s1, mu1, u1 = _setup_and_solve(D, p, tc_tiles=1, **kw)
    assert np.array_equal(u1, u2)
    ref = odd.solve(p, odd.Options(eps_rel=1e-6))
    assert close(u2, ref["u_eval"], 1e-8, "all-levels u, tiny")
