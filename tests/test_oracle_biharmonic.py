"""Pins of the oracle's biharmonic operator (the coupled system of Sec. 2.1:
Lap^2 u = f, u and Lap u given on the boundary, u and Lap u continuous across
the interface, both normal derivatives balanced), CPU only.

* the fourth-order feature rows against finite differences of lower ones;
* the two-component layout (multiplicities, numbering, per-component change
  of variables);
* the structured oracle against the literal dense brute force;
* exact recovery of a consistent coupled system;
* convergence to a manufactured solution as the networks grow.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ddelm, dense
from oracle.layout import Layout
from paper_2503_10032_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _lap_fd(fn, xy, h):
    f0 = fn(xy)
    return sum((fn(xy + h * e) - 2 * f0 + fn(xy - h * e)) / h ** 2 for e in np.eye(2))


def test_biharmonic_features_against_finite_differences():
    rng = np.random.default_rng(4)
    w = rng.uniform(-3, 3, (6, 2))
    b = rng.uniform(-1, 1, 6)
    xy = rng.uniform(0, 1, (9, 2))
    lap = ddelm.lap_phi(w, b, xy)
    np.testing.assert_allclose(lap, _lap_fd(lambda p: ddelm.phi(w, b, p), xy, 1e-4), rtol=1e-5, atol=1e-5)
    bil = ddelm.bilap_phi(w, b, xy)
    np.testing.assert_allclose(bil, _lap_fd(lambda p: ddelm.lap_phi(w, b, p), xy, 1e-4), rtol=1e-5,
                               atol=1e-5 * np.abs(bil).max())
    np.testing.assert_array_equal(ddelm.L_phi(w, b, xy, 2), bil)
    for nrm in ([1.0, 0.0], [0.0, -1.0]):
        n = np.tile([nrm], (9, 1))
        e = np.array(nrm)
        h = 1e-5
        fd = (ddelm.lap_phi(w, b, xy + h * e) - ddelm.lap_phi(w, b, xy - h * e)) / (2 * h)
        np.testing.assert_allclose(ddelm.F_lap_phi(w, b, xy, n), fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    comp = np.array([0, 1, 0, 1, 1, 0, 0, 1, 0])
    C = ddelm.C_rows(w, b, xy, comp)
    np.testing.assert_array_equal(C[comp == 0], ddelm.phi(w, b, xy[comp == 0]))
    np.testing.assert_array_equal(C[comp == 1], lap[comp == 1])


def test_two_component_layout():
    edge_pts = np.arange(4 * 4 + 5 * 3) % 3 + 2
    one = Layout(4, 3, (0.0, 2.0, 0.0, 1.0), edge_pts)
    two = Layout(4, 3, (0.0, 2.0, 0.0, 1.0), edge_pts, n_comp=2)
    assert (two.n_bnd, two.n_pi, two.n_delta) == (2 * one.n_bnd, 2 * one.n_pi, 2 * one.n_delta)
    cnt = np.zeros(two.n_gamma, np.int64)
    for s1, s2 in zip(one.subs, two.subs):
        np.add.at(cnt, s2.pi_gidx, 1)
        np.add.at(cnt, s2.dl_gidx, 1)
        kp, kd, kb = len(s1.pi_xy), len(s1.dl_xy), len(s1.bnd_xy)
        # component 0 keeps the one-component numbering shifted past the second Pi block
        np.testing.assert_array_equal(s2.pi_gidx[:kp], s1.pi_gidx)
        np.testing.assert_array_equal(s2.pi_gidx[kp:], s1.pi_gidx + one.n_pi)
        np.testing.assert_array_equal(s2.dl_gidx[:kd], s1.dl_gidx + one.n_pi)
        np.testing.assert_array_equal(s2.dl_gidx[kd:], s1.dl_gidx + one.n_pi + one.n_delta)
        np.testing.assert_array_equal(s2.bnd_gidx[kb:], s1.bnd_gidx + one.n_bnd)
        np.testing.assert_array_equal(s2.dl_comp, np.repeat([0, 1], kd))
        # the change of variables of a component-1 row refers to component-1 corners
        for k in range(kd, 2 * kd):
            for pi_idx in (s2.dl_alpha_pi[k], s2.dl_beta_pi[k]):
                if pi_idx >= 0:
                    assert s2.pi_comp[pi_idx] == 1
                    np.testing.assert_array_equal(s2.pi_xy[pi_idx], s1.pi_xy[pi_idx - kp])
    assert np.all(cnt[:two.n_pi] == 4) and np.all(cnt[two.n_pi:] == 2)


CASES = [(2, 2, 16, 50, 3, 1e-6, 0.999), (3, 3, 14, 50, 2, 1e-6, 0.5),
         (3, 2, 18, 60, 3, 0.0, 1.0), (3, 3, 14, 50, 2, 1e-6, 0.0), (2, 1, 14, 50, 3, 1e-6, 0.999)]


@pytest.mark.parametrize("case", CASES)
def test_biharmonic_structured_equals_dense_bruteforce(case):
    nx, ny, M, nI, e, eps, th = case
    p = inputs.small_problem(nx, ny, M=M, n_int=nI, edge_pts=e, n_rhs=2, op=inputs.OP_BIHARMONIC)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=eps, theta=th))
    mu, S, b = o.solve_direct()
    cs, mu_pi = o.reconstruct(mu)
    d = dense.solve_dense(o)
    assert _rel(S, d["S"]) < 1e-10
    assert _rel(b, d["b"]) < 1e-9
    assert _rel(mu, d["mu_delta"]) < 1e-9
    if o.n_pi:
        assert _rel(mu_pi, d["mu_pi"]) < 1e-9


def test_biharmonic_plain_flux_rows():
    """Plain A (Eq. (ddelm)) for the second component: a corner row is d Lap phi/dn
    at the corner with each of the two edges' outward normals, summed (times
    H^3, the weight of a third derivative)."""
    p = inputs.small_problem(3, 3, M=12, n_int=40, edge_pts=3, n_rhs=1, seed=9, op=inputs.OP_BIHARMONIC)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6, use_Am=False))
    L, sl = o.loc[4], o.lay.subs[4]
    kp = L.nPi // 2
    for k in range(kp, L.nPi):
        v = sl.pi_vertex[k]
        xy = o.lay.vxy(v)[None, :]
        nx_ = 1.0 if v[0] == 2 else -1.0
        ny_ = 1.0 if v[1] == 2 else -1.0
        H3 = (o.lay.hx * o.lay.hy) ** 1.5
        want = (ddelm.F_lap_phi(L.w, L.b, xy, np.array([[nx_, 0.0]])) +
                ddelm.F_lap_phi(L.w, L.b, xy, np.array([[0.0, ny_]]))) * H3
        np.testing.assert_allclose(L.Ahat[k], want[0], rtol=1e-13, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("theta", [0.0, 0.999])
def test_biharmonic_consistent_system_exact_recovery(theta):
    """A consistent biharmonic Eq. (ddelm) (c* in the null space of both continuity
    and both flux conditions) is solved exactly (ridge off)."""
    p = inputs.small_problem(3, 2, M=24, n_int=60, edge_pts=2, scale=2.0, seed=5, op=inputs.OP_BIHARMONIC)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=0.0, theta=theta))
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
    assert N.shape[1] > 0
    z = N @ np.random.default_rng(2).standard_normal(N.shape[1])
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
    cs, mu_pi = o.reconstruct(mu)
    assert _rel(mu[:, 0], mu_star[o.n_pi:]) < 1e-7
    assert _rel(mu_pi[:, 0], mu_star[:o.n_pi]) < 1e-7


def test_biharmonic_manufactured_solution_converges():
    """u = sin(pi x) sin(pi y) (Lap^2 u = 4 pi^4 u, Lap u = -2 pi^2 u on the
    boundary) and u = sin(2 pi x) cos(3 pi y): the error falls with M."""
    errs = []
    for M, nI, e, sc in ((60, 196, 8, 3.0), (150, 400, 14, 4.0)):
        p = inputs.make_problem(2, 2, M, nI, e, scale=sc, init="paper", seed=11,
                                solutions=[inputs._sin_sin(1, 1), inputs._sin2pix_cos3piy()],
                                op=inputs.OP_BIHARMONIC, points="grid")
        r = ddelm.solve(p, ddelm.Options(eps_rel=1e-8))
        errs.append(np.linalg.norm(r["u_eval"] - p.u_eval_exact, axis=0) / np.linalg.norm(p.u_eval_exact, axis=0))
    assert errs[1][0] < 1e-3 and errs[1][1] < 0.1
    assert np.all(errs[1] < 0.05 * errs[0])


def test_biharmonic_reweighting():
    """Every derivative of order k times H^k (H the subdomain size): interior
    rows H^4 Lap^2 phi with data H^4 f; the second component's boundary and
    continuity rows H^2 Lap phi with boundary data H^2 Lap u; flux rows
    H d phi/dn and H^3 d Lap phi/dn; point values unscaled.  A 3x2 grid on
    [0, 1.5] x [0, 1] has square subdomains of side H = 0.5."""
    p = inputs.make_problem(3, 2, 14, 50, 2, scale=3.0, init="uniform", seed=4, solutions=[inputs._sin_sin(1, 1)],
                            op=inputs.OP_BIHARMONIC, box=(0.0, 1.5, 0.0, 1.0), n_eval=8)
    o = ddelm.DDELMOracle(p, ddelm.Options(eps_rel=1e-6))
    s = 2.0   # 1 / H
    L, sl = o.loc[4], o.lay.subs[4]
    i0 = int(p.n_int[:4].sum())
    xI = p.x_int[i0:i0 + L.nI]
    np.testing.assert_allclose(L.K[:L.nI], ddelm.bilap_phi(L.w, L.b, xI) / s ** 4, rtol=1e-14, atol=0)
    kb = L.nB // 2
    np.testing.assert_allclose(L.K[L.nI:L.nI + kb], ddelm.phi(L.w, L.b, sl.bnd_xy[:kb]), rtol=1e-14, atol=0)
    np.testing.assert_allclose(L.K[L.nI + kb:L.nI + L.nB], ddelm.lap_phi(L.w, L.b, sl.bnd_xy[kb:]) / s ** 2,
                               rtol=1e-14, atol=0)
    kd = L.nDl // 2
    F0 = ddelm.F_phi(L.w, L.b, sl.dl_xy[:kd], sl.dl_normal[:kd]) / s
    F1 = ddelm.F_lap_phi(L.w, L.b, sl.dl_xy[kd:], sl.dl_normal[kd:]) / s ** 3
    np.testing.assert_allclose(L.Ahat[L.nPi:L.nPi + kd], F0, rtol=1e-14, atol=0)
    np.testing.assert_allclose(L.Ahat[L.nPi + kd:], F1, rtol=1e-14, atol=0)
    np.testing.assert_allclose(L.Kbar[L.m - kd:], F1, rtol=1e-14, atol=0)
    np.testing.assert_allclose(L.f[:L.nI, 0], p.f_int[i0:i0 + L.nI, 0] / s ** 4, rtol=1e-15, atol=0)
    np.testing.assert_allclose(L.f[L.nI + kb:L.nI + L.nB, 0], p.g_bnd[sl.bnd_gidx[kb:], 0] / s ** 2, rtol=1e-15,
                               atol=0)


def test_biharmonic_paper_scale_subdomains():
    """Subdomains of side 1/16 with the paper's l = 64 and 256 neurons (the
    16x16 case of Sec. 4.5), on a 4x4 patch: the reweighted system reaches a
    small error where unit weights do not (the Lap^2 phi rows are ~1e8 larger
    than the point values and, with the ridge, bury the continuity of u)."""
    p = inputs.make_problem(4, 4, 256, 400, 20, scale=64.0, init="paper", seed=2001,
                            solutions=[inputs._sin_sin(1, 1)], op=inputs.OP_BIHARMONIC, points="grid",
                            box=(0.0, 0.25, 0.0, 0.25))
    r = ddelm.solve(p, ddelm.Options(eps_rel=1e-8, theta=0.999))
    err = np.linalg.norm(r["u_eval"] - p.u_eval_exact) / np.linalg.norm(p.u_eval_exact)
    assert err < 1e-5, err
