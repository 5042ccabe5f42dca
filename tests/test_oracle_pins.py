"""Pins of the FP64 oracle to facts other than itself (CPU only).

* worked examples printed in the paper (T^i and A_m^i on a six-point edge);
* analytic feature derivatives against finite differences;
* the structured oracle against the literal dense brute force;
* exact recovery of a consistent coupled system by every variant;
* the Schur-complement solution against a library least-squares solve of the
  stacked system it is the normal equation of;
* symmetry and positive definiteness of S_theta and S_Pi;
* CG to a tight tolerance against the direct solve;
* a manufactured solution.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ddelm, dense
from oracle.layout import Layout
from paper_2503_10032_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#") / 5.0


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_T_matrix_worked_example():
    """Sec. 3.2: the layout's interpolation weights reproduce the printed T^i."""
    T_gold = _load("T_edge6.txt")
    lay = Layout(3, 3, (0.0, 1.0, 0.0, 1.0), np.full(24, 4))
    sl = lay.subs[4]                     # centre subdomain: every edge joins two cross points
    # bottom edge: its 4 Delta points come first among the local Delta points
    T = np.zeros((6, 6))
    T[0, 0] = T[5, 5] = 1.0
    for k in range(4):
        T[k + 1, k + 1] = 1.0
        T[k + 1, 0] = sl.dl_alpha[k]
        T[k + 1, 5] = sl.dl_beta[k]
    # the start vertex of the bottom edge is BL (local Pi 0), the end BR (local Pi 1)
    assert list(sl.dl_alpha_pi[:4]) == [0] * 4 and list(sl.dl_beta_pi[:4]) == [1] * 4
    np.testing.assert_allclose(T, T_gold, rtol=0, atol=1e-15)


def test_Tinv_rows_in_Kc():
    """K_c rows are (T^i)^{-1} C phi: T applied to them gives the point values back."""
    p = inputs.small_problem(3, 3, M=9, n_int=30, edge_pts=4, seed=3)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6))
    L, sl = o.loc[4], o.lay.subs[4]
    G = L.K[L.m - L.nG:]
    pt = ddelm.phi(L.w, L.b, np.vstack([sl.pi_xy, sl.dl_xy]))
    T = np.eye(L.nG)
    for k in range(L.nDl):
        T[L.nPi + k, sl.dl_alpha_pi[k]] += sl.dl_alpha[k]
        T[L.nPi + k, sl.dl_beta_pi[k]] += sl.dl_beta[k]
    np.testing.assert_allclose(T @ G, pt, rtol=0, atol=1e-14)


def test_Am_worked_example():
    """Sec. 3.2: per edge, a corner row is the mean flux with the opposing corner left out."""
    Am_gold = _load("Am_edge6.txt")
    lay = Layout(3, 3, (0.0, 1.0, 0.0, 1.0), np.full(24, 4))
    sl = lay.subs[4]
    edge_pts = [lay.vxy((1, 1)) + k / 5 * (lay.vxy((2, 1)) - lay.vxy((1, 1))) for k in range(6)]
    nb = np.array([0.0, -1.0])          # outward normal of the bottom edge
    for row, pi_local in ((0, 0), (5, 1)):
        terms = [(w, xy) for w, xy, n in sl.am_terms[pi_local] if np.allclose(n, nb)]
        weights = np.zeros(6)
        for w, xy in terms:
            j = int(np.argmin([np.linalg.norm(xy - e) for e in edge_pts]))
            assert np.linalg.norm(xy - edge_pts[j]) < 1e-14
            weights[j] += w
        np.testing.assert_allclose(weights, Am_gold[row], rtol=0, atol=1e-15)
        # each cross point also sums the mean flux of the subdomain's other incident edge
        assert len(sl.am_terms[pi_local]) == 2 * 5


@pytest.mark.parametrize("op", [0, 1])
def test_features_against_finite_differences(op):
    rng = np.random.default_rng(0)
    w = rng.uniform(-3, 3, (5, 2))
    b = rng.uniform(-1, 1, 5)
    xy = rng.uniform(0, 1, (7, 2))
    h = 1e-4
    f0 = ddelm.phi(w, b, xy)
    fx = [(ddelm.phi(w, b, xy + h * e) - ddelm.phi(w, b, xy - h * e)) / (2 * h) for e in np.eye(2)]
    lap = sum((ddelm.phi(w, b, xy + h * e) - 2 * f0 + ddelm.phi(w, b, xy - h * e)) / h ** 2 for e in np.eye(2))
    a = 1.0 + 0.3 * xy[:, 0]
    ga = np.stack([0.3 * np.ones(7), np.zeros(7)], 1)
    L = ddelm.L_phi(w, b, xy, op, a, ga)
    ref = -lap if op == 0 else -(a[:, None] * lap + ga[:, :1] * fx[0] + ga[:, 1:] * fx[1])
    np.testing.assert_allclose(L, ref, rtol=1e-5, atol=1e-5)
    n = np.tile([[0.0, -1.0]], (7, 1))
    np.testing.assert_allclose(ddelm.F_phi(w, b, xy, n), -fx[1], rtol=1e-7, atol=1e-7)


def test_layout_multiplicities():
    """Every Delta point lies on two subdomains, every Pi point on four (Sec. 3)."""
    lay = Layout(4, 3, (0.0, 2.0, 0.0, 1.0), np.arange(4 * 4 + 5 * 3) % 3 + 2)
    cnt = np.zeros(lay.n_gamma, np.int64)
    for sl in lay.subs:
        np.add.at(cnt, sl.pi_gidx, 1)
        np.add.at(cnt, sl.dl_gidx, 1)
    assert np.all(cnt[:lay.n_pi] == 4) and np.all(cnt[lay.n_pi:] == 2)
    bcnt = np.zeros(lay.n_bnd, np.int64)
    for sl in lay.subs:
        np.add.at(bcnt, sl.bnd_gidx, 1)
    assert np.all(bcnt >= 1)
    xb = inputs.boundary_points(4, 3, (0.0, 2.0, 0.0, 1.0), lay.edge_pts)
    for sl in lay.subs:
        np.testing.assert_allclose(xb[sl.bnd_gidx], sl.bnd_xy, atol=1e-15)


CASES = [(2, 2, 12, 40, 3, 1e-6, 0.999), (3, 3, 10, 40, 2, 1e-6, 0.5),
         (3, 2, 14, 50, 4, 0.0, 1.0), (2, 1, 10, 40, 3, 1e-6, 0.999),
         (3, 3, 10, 40, 2, 1e-6, 0.0)]


@pytest.mark.parametrize("case", CASES)
def test_structured_equals_dense_bruteforce(case):
    nx, ny, M, nI, e, eps, th = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=2)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=eps, theta=th))
    mu, S, b = o.solve_direct()
    cs, mu_pi = o.reconstruct(mu)
    d = dense.solve_dense(o)
    assert _rel(S, d["S"]) < 1e-11
    assert _rel(b, d["b"]) < 1e-10
    assert _rel(mu, d["mu_delta"]) < 1e-10
    if o.n_pi:
        assert _rel(mu_pi, d["mu_pi"]) < 1e-10
    assert _rel(np.concatenate(cs), np.concatenate(d["c"])) < 1e-10


@pytest.mark.parametrize("theta", [0.0, 1.0])
def test_plain_flux_rows(theta):
    """The plain flux rows A of Eq. (ddelm) (no A_m): a corner's row is the flux at
    the corner with each of the two edges' outward normals, summed (the corner
    normal is undefined); its Delta rows are the A_m Delta rows; and the
    structured method with these rows equals the dense brute force."""
    p = inputs.small_problem(3, 3, M=12, n_int=40, edge_pts=3, n_rhs=1, seed=9)
    o_a = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=theta, use_Am=False))
    o_m = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=theta))
    for i, (La, Lm) in enumerate(zip(o_a.loc, o_m.loc)):
        sl = o_a.lay.subs[i]
        np.testing.assert_array_equal(La.Ahat[La.nPi:], Lm.Ahat[Lm.nPi:])
        for k, v in enumerate(sl.pi_vertex):
            xy = o_a.lay.vxy(v)[None, :]
            ix, iy = i % p.nx, i // p.nx
            # the two edges of subdomain i meeting corner v: a vertical one (normal +-x), a horizontal one (+-y)
            nx_ = 1.0 if v[0] == ix + 1 else -1.0
            ny_ = 1.0 if v[1] == iy + 1 else -1.0
            want = ddelm.F_phi(La.w, La.b, xy, np.array([[nx_, 0.0]])) + \
                ddelm.F_phi(La.w, La.b, xy, np.array([[0.0, ny_]]))
            np.testing.assert_allclose(La.Ahat[k], want[0], rtol=1e-13, atol=1e-13)
    mu, S, b = o_a.solve_direct()
    d = dense.solve_dense(o_a)
    assert _rel(S, d["S"]) < 1e-11
    assert _rel(mu, d["mu_delta"]) < 1e-10
    assert _rel(S, o_m.assemble_S_theta()) > 1e-6   # the modification changes the operator


def test_normal_equation_is_stacked_least_squares():
    """Eq. (nn-mixed) + Eq. (coarse_sol_2) minimise |K~ c + B~ mu - f~|^2 + |W^1/2 (D~ mu - d~)|^2."""
    p = inputs.small_problem(3, 3, M=10, n_int=40, edge_pts=2, n_rhs=1, seed=11)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=0.9))
    d = dense.solve_dense(o)
    Wh = sla.sqrtm(d["W"]).real
    Kt, Bt = d["Kt"], d["Bt"]
    top = np.hstack([Kt, Bt])
    bot = np.hstack([np.zeros((Wh.shape[0], Kt.shape[1])), Wh @ d["Dt"]])
    sol = np.linalg.lstsq(np.vstack([top, bot]), np.vstack([d["ft"], Wh @ d["dt"]]), rcond=None)[0]
    mu = sol[Kt.shape[1]:]
    mu_o, _, _ = o.solve_direct()
    assert _rel(mu_o, mu) < 1e-9


@pytest.mark.parametrize("theta", [0.0, 0.999, 1.0])
def test_consistent_system_exact_recovery(theta):
    """A consistent Eq. (ddelm) is solved exactly by every variant (ridge off)."""
    p = inputs.small_problem(3, 2, M=16, n_int=60, edge_pts=3, scale=4.0, seed=5)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=0.0, theta=theta))
    g = dense.global_system(o)
    nc, nG = g["K"].shape[1], g["B"].shape[1]
    # constraints: Gamma rows of K c + B mu = 0 and A c = 0
    rows = []
    r0 = 0
    for L in o.loc:
        M = L.K.shape[1]
        sel = np.zeros((L.nG, g["K"].shape[0]))
        sel[np.arange(L.nG), r0 + L.m - L.nG + np.arange(L.nG)] = 1.0
        rows.append(sel)
        r0 += L.m + M
    SelG = np.vstack(rows)
    C = np.vstack([np.hstack([SelG @ g["K"], SelG @ g["B"]]),
                   np.hstack([g["A"], np.zeros((nG, nG))])])
    N = sla.null_space(C)
    assert N.shape[1] > 0
    z = N @ np.random.default_rng(1).standard_normal(N.shape[1])
    c_star, mu_star = z[:nc], z[nc:]
    # right-hand side f = K c* on the interior/boundary rows
    off_c = 0
    for L in o.loc:
        M = L.K.shape[1]
        nIB = L.m - L.nG
        L.f = np.zeros((L.m, 1))
        L.f[:nIB, 0] = L.K[:nIB] @ c_star[off_c:off_c + M]
        off_c += M
    o._build_coarse()
    mu, _, _ = o.solve_direct()
    cs, mu_pi = o.reconstruct(mu)
    assert _rel(mu[:, 0], mu_star[o.n_pi:]) < 1e-8
    assert _rel(mu_pi[:, 0], mu_star[:o.n_pi]) < 1e-8
    # c is only as well determined as cond(K^i) allows (M = 16 features at scale 4)
    assert _rel(np.concatenate(cs)[:, 0], c_star) < 1e-6


def test_theta_zero_is_coarse_space_system():
    """theta = 0 turns Eq. (nn-mixed) into Eq. (coarse_sol_1); theta = 1 into Eq. (nn)."""
    p = inputs.small_problem(3, 3, M=10, n_int=40, edge_pts=2, seed=2)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=0.0))
    d = dense.solve_dense(o)
    Dt, Bt, Kt = d["Dt"], d["Bt"], d["Kt"]
    S_cs = Bt.T @ Bt + Dt.T @ Dt - Bt.T @ Kt @ np.linalg.pinv(Kt) @ Bt
    assert _rel(o.assemble_S_theta(), S_cs) < 1e-11
    o.o.theta = 1.0
    d1 = dense.solve_dense(o)
    S_nn = Bt.T @ Bt + Dt.T @ d1["P"].T @ d1["P"] @ Dt - Bt.T @ Kt @ np.linalg.pinv(Kt) @ Bt
    assert _rel(o.assemble_S_theta(), S_nn) < 1e-11


def test_no_cross_points_is_vanilla_ddelm():
    """With Pi empty (one row of subdomains) the system is the Sec. 2.2.1 Schur complement."""
    p = inputs.small_problem(3, 1, M=12, n_int=40, edge_pts=3, seed=4)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=0.0))
    assert o.n_pi == 0
    g = dense.global_system(o)
    K, B, A, f = g["K"], g["B"], g["A"], g["f"]
    Kp = np.linalg.pinv(K)
    D, dd = -A @ Kp @ B, -A @ Kp @ f
    S = B.T @ B + D.T @ D - B.T @ K @ Kp @ B
    rhs = (B.T - B.T @ K @ Kp) @ f + D.T @ dd
    mu, S_o, b_o = o.solve_direct()
    assert _rel(S_o, S) < 1e-11 and _rel(b_o, rhs) < 1e-10
    cs, _ = o.reconstruct(mu)
    c_ref = Kp @ (f - B @ mu)
    assert _rel(np.concatenate(cs), c_ref) < 1e-9


@pytest.mark.parametrize("op", [0, 2])
def test_vanilla_ddelm_with_cross_points(op):
    """use_coarse = False (vanilla DDELM, Sec. 2.2.1): every cross point is an
    interface unknown of its four subdomains, with the plain corner flux rows;
    the structured system equals the literal Eq. (schur) Schur complement."""
    p = inputs.small_problem(3, 3, M=30, n_int=90, edge_pts=3, seed=5, op=op)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, theta=0.0, use_coarse=False))
    nc = 2 if op == 2 else 1
    assert o.n_pi == 0 and o.n_dl == nc * (4 + 12 * 3)
    cnt = np.zeros(o.n_dl, np.int64)
    for L in o.loc:
        np.add.at(cnt, L.gdl, 1)
    assert sorted(set(cnt.tolist())) == [2, 4] and (cnt == 4).sum() == 4 * nc
    # the centre subdomain's corner rows: the flux with each edge's outward normal, summed
    L, sl = o.loc[4], o.lay.subs[4]
    for k in range(4):
        xy = sl.dl_xy[k:k + 1]
        nrm = sl.dl_normal[k]
        assert abs(nrm[0]) == 1.0 and abs(nrm[1]) == 1.0
        want = ddelm.F_phi(L.w, L.b, xy, np.array([[nrm[0], 0.0]])) + \
            ddelm.F_phi(L.w, L.b, xy, np.array([[0.0, nrm[1]]]))
        if op == 2:
            want = want / 3.0      # the biharmonic flux weight H (subdomains of side 1/3)
        np.testing.assert_allclose(L.Ahat[k], want[0], rtol=1e-12, atol=1e-13 * np.abs(want).max())
    g = dense.global_system(o)
    K, B, A, f = g["K"], g["B"], g["A"], g["f"]
    Kp = np.linalg.pinv(K)
    D, dd = -A @ Kp @ B, -A @ Kp @ f
    S = B.T @ B + D.T @ D - B.T @ K @ Kp @ B
    rhs = (B.T - B.T @ K @ Kp) @ f + D.T @ dd
    mu, S_o, b_o = o.solve_direct()
    assert _rel(S_o, S) < 1e-10 and _rel(b_o, rhs) < 1e-10
    cs, _ = o.reconstruct(mu)
    assert _rel(np.concatenate(cs), Kp @ (f - B @ mu)) < 1e-8


def test_vanilla_consistent_system_exact_recovery():
    """A consistent Eq. (ddelm) on a grid with cross points is solved exactly by
    vanilla DDELM (ridge off)."""
    p = inputs.small_problem(3, 2, M=16, n_int=60, edge_pts=3, scale=4.0, seed=5)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=0.0, theta=0.0, use_coarse=False))
    g = dense.global_system(o)
    nc, nG = g["K"].shape[1], g["B"].shape[1]
    rows, r0 = [], 0
    for L in o.loc:
        M = L.K.shape[1]
        sel = np.zeros((L.nG, g["K"].shape[0]))
        sel[np.arange(L.nG), r0 + L.m - L.nG + np.arange(L.nG)] = 1.0
        rows.append(sel)
        r0 += L.m + M
    SelG = np.vstack(rows)
    C = np.vstack([np.hstack([SelG @ g["K"], SelG @ g["B"]]), np.hstack([g["A"], np.zeros((nG, nG))])])
    N = sla.null_space(C)
    z = N @ np.random.default_rng(3).standard_normal(N.shape[1])
    c_star, mu_star = z[:nc], z[nc:]
    off_c = 0
    for L in o.loc:
        M = L.K.shape[1]
        nIB = L.m - L.nG
        L.f = np.zeros((L.m, 1))
        L.f[:nIB, 0] = L.K[:nIB] @ c_star[off_c:off_c + M]
        off_c += M
    o._build_coarse()
    mu, _, _ = o.solve_direct()
    assert _rel(mu[:, 0], mu_star) < 1e-8


def test_symmetric_positive_definite():
    p = inputs.small_problem(3, 3, M=12, n_int=50, edge_pts=3, seed=9)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-8))
    S = o.assemble_S_theta()
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
    assert np.abs(o.S_Pi - o.S_Pi.T).max() < 1e-12 * np.abs(o.S_Pi).max()
    assert np.linalg.eigvalsh(o.S_Pi).min() > 0


def test_cg_matches_direct():
    p = inputs.small_problem(3, 3, M=12, n_int=50, edge_pts=3, seed=9, n_rhs=2)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-8))
    mu, _, _ = o.solve_direct()
    mu_cg, it = o.solve_cg(tol=1e-13)
    assert it > 0 and _rel(mu_cg, mu) < 1e-10


def test_manufactured_solution_2x2():
    """Sanity: the 2x2, M=100 Poisson problem is solved to a small error."""
    p = inputs.config("poisson_2x2_m100")
    r = ddelm.solve(p, ddelm.Options(eps_rel=1e-8), method="cg")
    err = _rel(r["u_eval"], p.u_eval_exact)
    assert err < 1e-4, err
    assert r["iters"] < 100
