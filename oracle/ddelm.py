"""Structured FP64 DDELM-NN oracle (test infrastructure only).

Every step follows the paper's equations in the paper's order and notation;
numpy's Householder QR and Cholesky serve as the library steps.  Parity of the
CUDA path is checked against the quantities returned here.

Method (Sec. 2.2.1, Sec. 3, Sec. 3.1, Sec. 3.2):

* local matrices (Sec. 2.2.1 and Sec. 3.2): K_c^i = [L phi(x_I); B phi(x_B);
  (T^i)^{-1} C phi(x_Gamma^i)], B^i = [0; 0; -R^i], A_m^i (flux rows, corner
  rows replaced by mean edge flux), f^i = [f(x_I); g(x_B); 0];
* Neumann matrices (Sec. 3.1): K-bar^i = [L phi(x_I); B phi(x_B); C phi(x_Pi);
  F phi(x_Delta)], B-bar^i = [0; 0; 0; -R_f^i], A-bar^i = C phi^i(x_Delta);
* D_ab = -A_a K^+ B_b and d_a = -A_a K^+ f summed over subdomains (Sec. 3);
* S_Pi = B_Pi^T B_Pi + D_PiPi^T D_PiPi - B_Pi^T K K^+ B_Pi, assembled in full and
  Cholesky-factored (Sec. 3); application of K~^+ and of (K~^+)^T (Sec. 3);
* D~ = -A~ K~^+ B~, d~ = -A~ K~^+ f~, P = A-bar K-bar^+ B-bar,
  W = theta P^T P + (1 - theta) I and the mixed system Eq. (nn-mixed);
* [c; mu_Pi] = K~^+ (f~ - B~ mu_Delta), Eq. (coarse_sol_2).

Readings where the paper is silent:

* the local least-squares problems carry a ridge term: K^+ v is the minimiser
  of |K c - v|^2 + eps^2 |c|^2 with eps^2 = eps_rel^2 |K|_F^2 / M, i.e. K^+ is
  the pseudo-inverse of K augmented by rows eps*I with zero data (the same for
  K-bar with its own eps); eps_rel = 0 gives the Moore-Penrose pseudo-inverse;
* F phi = (w . n) (1 - tanh^2) with n the subdomain's outward normal; for the
  diffusion operator the flux is the normal derivative as well;
* A-bar^i uses the same rows as the Delta rows of K_c^i (the (T^i)^{-1} C phi
  rows) when the change of variables is on;
* R_f^i is the plain restriction (no sign), as for R^i;
* biharmonic (op 2, the coupled system of Sec. 2.1): every boundary and
  interface point carries two components (`layout.Layout(n_comp=2)`), u and
  v = H^2 Lap u.  The loss terms are reweighted (Sec. 1 announces a
  reweighting and never gives it) by writing every derivative of order k
  times H^k, H = sqrt(hx hy) the subdomain size: interior rows H^4 Lap^2 phi
  with data H^4 f, boundary rows phi and H^2 Lap phi with data g_1 and
  H^2 g_2, continuity rows phi and H^2 Lap phi, flux rows H d phi/dn and
  H^3 d Lap phi/dn; mu of component 1 is v.  The change of variables and A_m
  act on each component separately;
* vanilla DDELM (`Options.use_coarse = False`, Sec. 2.2.1): no coarse space;
  every cross point is an interface unknown of the Delta set shared by its
  four subdomains, with the plain corner flux row (the sum of the fluxes
  with the two edge normals of the subdomain there).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .layout import Layout


@dataclasses.dataclass
class Options:
    theta: float = 0.999           # Eq. (nn-mixed); 0.999 in Sec. 4.2.2
    eps_rel: float = 1e-8          # ridge reading (module docstring)
    use_change_of_vars: bool = True  # K_c instead of K (Sec. 3.2)
    use_Am: bool = True             # A_m instead of the plain flux rows A (Sec. 3.2)
    use_coarse: bool = True         # False: vanilla DDELM (Sec. 2.2.1), cross points in Delta, Pi empty
    tol: float = 1e-9              # CG relative residual (Sec. 4)
    max_iters: int = 20000


# ----------------------------------------------------------------------------
# features of phi_j(x) = tanh(w_j . x + b_j)  (Sec. 2.2)
# ----------------------------------------------------------------------------

def _z(w, b, xy):
    return xy @ w.T + b[None, :]


def phi(w, b, xy):
    """C phi = B phi = phi = tanh(w.x + b)."""
    return np.tanh(_z(w, b, xy))


def L_phi(w, b, xy, op, a=None, grad_a=None):
    """L phi for -Lap (op 0), -div(a grad) (op 1) or Lap^2 (op 2).

    With t = tanh(z): grad phi = w (1 - t^2), Lap phi = |w|^2 (-2 t (1 - t^2)).
    -div(a grad phi) = -a Lap phi - grad a . grad phi.
    """
    if op == 2:
        return bilap_phi(w, b, xy)
    t = np.tanh(_z(w, b, xy))
    s1 = 1.0 - t * t
    w2 = (w * w).sum(1)[None, :]
    lap = -2.0 * w2 * t * s1
    if op == 0:
        return -lap
    return -a[:, None] * lap - (grad_a @ w.T) * s1


# Derivatives of tanh as polynomials in t = tanh z (d^k/dz^k tanh, k = 1..4):
#   1 - t^2,  -2 t (1 - t^2),  -2 (1 - t^2)(1 - 3 t^2),  8 t (1 - t^2)(2 - 3 t^2).
# For phi_j(x) = tanh(w_j . x + b_j): Lap phi = |w|^2 times the second,
# grad Lap phi = |w|^2 w times the third, Lap^2 phi = |w|^4 times the fourth.

def lap_phi(w, b, xy):
    """Lap phi (the second derivative of tanh times |w|^2)."""
    t = np.tanh(_z(w, b, xy))
    w2 = (w * w).sum(1)[None, :]
    return -2.0 * w2 * t * (1.0 - t * t)


def F_lap_phi(w, b, xy, normals):
    """d(Lap phi)/dn (the third derivative of tanh times |w|^2 (w . n))."""
    t = np.tanh(_z(w, b, xy))
    w2 = (w * w).sum(1)[None, :]
    return -2.0 * w2 * (1.0 - t * t) * (1.0 - 3.0 * t * t) * (normals @ w.T)


def bilap_phi(w, b, xy):
    """Lap^2 phi (the fourth derivative of tanh times |w|^4)."""
    t = np.tanh(_z(w, b, xy))
    w2 = (w * w).sum(1)[None, :]
    return 8.0 * w2 * w2 * t * (1.0 - t * t) * (2.0 - 3.0 * t * t)


def F_phi(w, b, xy, normals):
    """F phi = d phi / dn = (w . n)(1 - t^2)."""
    t = np.tanh(_z(w, b, xy))
    return (normals @ w.T) * (1.0 - t * t)


def C_rows(w, b, xy, comp, w_c1=1.0):
    """Continuity / boundary rows: phi for component 0, w_c1 Lap phi for component 1."""
    out = phi(w, b, xy)
    one = np.asarray(comp) == 1
    if one.any():
        out[one] = w_c1 * lap_phi(w, b, xy[one])
    return out


def F_rows(w, b, xy, normals, comp, w_f=(1.0, 1.0)):
    """Flux rows: w_f[0] d phi/dn for component 0, w_f[1] d Lap phi/dn for component 1."""
    out = w_f[0] * F_phi(w, b, xy, normals)
    one = np.asarray(comp) == 1
    if one.any():
        out[one] = w_f[1] * F_lap_phi(w, b, xy[one], normals[one])
    return out


# ----------------------------------------------------------------------------

class _Local:
    pass


def _ridge_pinv(K, eps_rel):
    """K^+ of the ridge reading: pinv of [K; eps I], columns of the K rows.

    Householder QR of the augmented matrix (numpy/LAPACK), K^+ = R^{-1} Q_1^T.
    """
    m, M = K.shape
    eps2 = eps_rel ** 2 * float((K * K).sum()) / M
    Kaug = np.vstack([K, np.sqrt(eps2) * np.eye(M)])
    Q, R = np.linalg.qr(Kaug)
    pinv = sla.solve_triangular(R, Q.T, lower=False)
    return pinv[:, :m], eps2


class DDELMOracle:
    """The structured oracle.  ``prob`` is a problem in the plain-array format."""

    def __init__(self, prob, opts: Options | None = None, only=None):
        """only: optional list of subdomains; builds just their local blocks and
        skips the coarse problem (used to time a bounded sample of the setup)."""
        self.p = prob
        self.o = opts or Options()
        self.lay = Layout(prob.nx, prob.ny, prob.box, prob.edge_pts, use_Am=self.o.use_Am,
                          n_comp=2 if prob.op == 2 else 1, use_coarse=self.o.use_coarse)
        self.n_pi, self.n_dl = self.lay.n_pi, self.lay.n_delta
        self._build_local(only)
        if only is None:
            self._build_coarse()

    # ------------------------------------------------------------ local
    def _build_local(self, only=None):
        p, o = self.p, self.o
        Moff = np.concatenate([[0], np.cumsum(p.M)])
        Ioff = np.concatenate([[0], np.cumsum(p.n_int)])
        self.loc = []
        for i, sl in enumerate(self.lay.subs):
            if only is not None and i not in only:
                self.loc.append(None)
                continue
            L = _Local()
            w = p.scale * p.w_hat[Moff[i]:Moff[i + 1]]
            b = p.scale * p.b_hat[Moff[i]:Moff[i + 1]]
            L.w, L.b = w, b
            xI = p.x_int[Ioff[i]:Ioff[i + 1]]
            aI = p.a_int[Ioff[i]:Ioff[i + 1]]
            gI = p.grad_a_int[Ioff[i]:Ioff[i + 1]]
            # biharmonic: every derivative of order k times H^k (module docstring)
            H = np.sqrt(self.lay.hx * self.lay.hy)
            bih = p.op == 2
            w_int = H ** 4 if bih else 1.0
            w_c1 = H ** 2 if bih else 1.0
            w_f = (H, H ** 3) if bih else (1.0, 1.0)
            rows_I = w_int * L_phi(w, b, xI, p.op, aI, gI)
            rows_B = C_rows(w, b, sl.bnd_xy, sl.bnd_comp, w_c1)
            C_pi = C_rows(w, b, sl.pi_xy, sl.pi_comp, w_c1)
            C_dl = C_rows(w, b, sl.dl_xy, sl.dl_comp, w_c1)
            if o.use_change_of_vars:
                # (T^i)^{-1} C phi: Delta row minus its weights on the corner rows
                Tinv_dl = C_dl.copy()
                for k in range(len(sl.dl_xy)):
                    if sl.dl_alpha_pi[k] >= 0:
                        Tinv_dl[k] -= sl.dl_alpha[k] * C_pi[sl.dl_alpha_pi[k]]
                    if sl.dl_beta_pi[k] >= 0:
                        Tinv_dl[k] -= sl.dl_beta[k] * C_pi[sl.dl_beta_pi[k]]
            else:
                Tinv_dl = C_dl
            L.nI, L.nB, L.nPi, L.nDl = len(xI), len(sl.bnd_xy), len(sl.pi_xy), len(sl.dl_xy)
            L.nG = L.nPi + L.nDl
            L.K = np.vstack([rows_I, rows_B, C_pi, Tinv_dl])
            L.m = L.K.shape[0]
            # A_m^i: Delta rows are point fluxes, Pi rows the mean edge fluxes
            F_dl = F_rows(w, b, sl.dl_xy, sl.dl_normal, sl.dl_comp, w_f)
            A_pi = np.zeros((L.nPi, len(w)))
            for k, terms in enumerate(sl.am_terms):
                for wgt, xy, nrm in terms:
                    A_pi[k] += wgt * F_rows(w, b, xy[None, :], np.array([nrm]), [sl.pi_comp[k]], w_f)[0]
            L.Ahat = np.vstack([A_pi, F_dl])
            L.Kbar = np.vstack([rows_I, rows_B, C_pi, F_dl])
            L.Abar = Tinv_dl
            g_w = np.where(np.asarray(sl.bnd_comp) == 1, w_c1, 1.0)[:, None]
            L.f = np.vstack([w_int * p.f_int[Ioff[i]:Ioff[i + 1]], g_w * p.g_bnd[sl.bnd_gidx],
                             np.zeros((L.nG, p.n_rhs))])
            L.gpi = sl.pi_gidx                       # R_Pi^i as an index map
            L.gdl = sl.dl_gidx - self.n_pi           # R_Delta^i (= R_f^i) as an index map
            L.Kpinv, L.eps2 = _ridge_pinv(L.K, o.eps_rel)
            L.Kbar_pinv, L.eps2_bar = _ridge_pinv(L.Kbar, o.eps_rel)
            self.loc.append(L)

    # ------------------------------------------------------------ B, A maps
    # B_b mu_b on subdomain i is supported on the Gamma rows: -(R_b^i mu_b).
    def _B_gamma(self, L, mu_pi=None, mu_dl=None, k=1):
        g = np.zeros((L.nG, k))
        if mu_pi is not None and L.nPi:
            g[:L.nPi] -= mu_pi[L.gpi]
        if mu_dl is not None and L.nDl:
            g[L.nPi:] -= mu_dl[L.gdl]
        return g

    def _full_m(self, L, gam, k):
        v = np.zeros((L.m, k))
        v[L.m - L.nG:] = gam
        return v

    def B_T(self, vs):
        """(B_Pi^T v, B_Delta^T v) for per-subdomain m-vectors v."""
        k = vs[0].shape[1]
        out_pi, out_dl = np.zeros((self.n_pi, k)), np.zeros((self.n_dl, k))
        for L, v in zip(self.loc, vs):
            g = v[L.m - L.nG:]
            np.add.at(out_pi, L.gpi, -g[:L.nPi])
            np.add.at(out_dl, L.gdl, -g[L.nPi:])
        return out_pi, out_dl

    def A_apply(self, cs):
        """(A_Pi c, A_Delta c) = sum_i R^i^T A_m^i c^i."""
        k = cs[0].shape[1]
        out_pi, out_dl = np.zeros((self.n_pi, k)), np.zeros((self.n_dl, k))
        for L, c in zip(self.loc, cs):
            r = L.Ahat @ c
            np.add.at(out_pi, L.gpi, r[:L.nPi])
            np.add.at(out_dl, L.gdl, r[L.nPi:])
        return out_pi, out_dl

    def A_T(self, y_pi, y_dl):
        """A^T [y_Pi; y_Delta] -> per-subdomain c-space vectors."""
        out = []
        for L in self.loc:
            k = (y_pi if y_pi is not None else y_dl).shape[1]
            loc = np.zeros((L.nG, k))
            if y_pi is not None:
                loc[:L.nPi] = y_pi[L.gpi]
            if y_dl is not None:
                loc[L.nPi:] = y_dl[L.gdl]
            out.append(L.Ahat.T @ loc)
        return out

    # ------------------------------------------------------------ coarse (Sec. 3)
    def _build_coarse(self):
        npi, ndl = self.n_pi, self.n_dl
        # D_ab = -A_a K^+ B_b: evaluated column by column on unit vectors of b
        self.D_PiPi = np.zeros((npi, npi))
        self.D_PiDl = np.zeros((npi, ndl))
        for L in self.loc:
            KpB = L.Kpinv[:, L.m - L.nG:]            # K^+ restricted to the Gamma rows
            blk = -(L.Ahat @ KpB) @ (-np.eye(L.nG))   # -A^i K^+ B^i on local Gamma
            ii = L.gpi
            self.D_PiPi[np.ix_(ii, ii)] += blk[:L.nPi, :L.nPi]
            self.D_PiDl[np.ix_(ii, L.gdl)] += blk[:L.nPi, L.nPi:]
        # d_a = -A_a K^+ f
        ys = [L.Kpinv @ L.f for L in self.loc]
        d_pi, d_dl = self.A_apply(ys)
        self.d_pi = -d_pi
        # S_Pi = B_Pi^T B_Pi + D_PiPi^T D_PiPi - B_Pi^T K K^+ B_Pi
        S = self.D_PiPi.T @ self.D_PiPi
        for L in self.loc:
            ii = L.gpi
            Epi = np.zeros((L.m, L.nPi))
            Epi[L.m - L.nG + np.arange(L.nPi), np.arange(L.nPi)] = -1.0   # B_Pi^i columns
            KKB = L.K @ (L.Kpinv @ Epi)
            S[np.ix_(ii, ii)] += Epi.T @ Epi - Epi.T @ KKB
        self.S_Pi = S
        self.S_Pi_chol = np.linalg.cholesky(S) if npi else np.zeros((0, 0))

    def _S_Pi_solve(self, r):
        if self.n_pi == 0:
            return np.zeros((0, r.shape[1]))
        return sla.cho_solve((self.S_Pi_chol, True), r)

    # K~^+ [phi; psi] (Sec. 3): per-subdomain m-vectors phi, |Pi|-vector psi
    def Kt_pinv(self, phis, psi):
        k = phis[0].shape[1]
        bpi, _ = self.B_T(phis)                                   # B_Pi^T phi
        kk = [L.K @ (L.Kpinv @ ph) for L, ph in zip(self.loc, phis)]
        bkk, _ = self.B_T(kk)                                     # B_Pi^T K K^+ phi
        mu_pi = self._S_Pi_solve(bpi - bkk + self.D_PiPi.T @ psi)
        cs = [L.Kpinv @ (ph - self._full_m(L, self._B_gamma(L, mu_pi=mu_pi, k=k), k))
              for L, ph in zip(self.loc, phis)]
        return cs, mu_pi

    def Kt_apply(self, cs, mu_pi):
        """K~ [c; mu_Pi] = [K c + B_Pi mu_Pi; D_PiPi mu_Pi]."""
        k = cs[0].shape[1]
        ms = [L.K @ c + self._full_m(L, self._B_gamma(L, mu_pi=mu_pi, k=k), k)
              for L, c in zip(self.loc, cs)]
        return ms, self.D_PiPi @ mu_pi

    # (K~^+)^T [phi; 0] (Sec. 3), phi per-subdomain c-space vectors
    def Kt_pinvT_phi0(self, phis):
        k = phis[0].shape[1]
        KpT = [L.Kpinv.T @ ph for L, ph in zip(self.loc, phis)]  # (K^+)^T phi
        bpi, _ = self.B_T(KpT)
        nu = self._S_Pi_solve(-bpi)
        out = []
        for L, v in zip(self.loc, KpT):
            Bnu = self._full_m(L, self._B_gamma(L, mu_pi=nu, k=k), k)
            out.append(v - L.K @ (L.Kpinv @ Bnu) + Bnu)
        return out, self.D_PiPi @ nu

    # B~ mu_Delta = [B_Delta mu_Delta; D_PiDelta mu_Delta]
    def Bt_apply(self, mu_dl):
        k = mu_dl.shape[1]
        ms = [self._full_m(L, self._B_gamma(L, mu_dl=mu_dl, k=k), k) for L in self.loc]
        return ms, self.D_PiDl @ mu_dl

    def Bt_T(self, ms, v_pi):
        """B~^T [v; v_Pi] = B_Delta^T v + D_PiDelta^T v_Pi."""
        _, bdl = self.B_T(ms)
        return bdl + self.D_PiDl.T @ v_pi

    # ------------------------------------------------------------ D~, P (Sec. 3, 3.1)
    def Dt_apply(self, mu_dl):
        """D~ mu = -A~ K~^+ B~ mu, A~ = [A_Delta 0]."""
        ms, psi = self.Bt_apply(mu_dl)
        cs, _ = self.Kt_pinv(ms, psi)
        _, adl = self.A_apply(cs)
        return -adl

    def Dt_T(self, y):
        """D~^T y = -B~^T (K~^+)^T A~^T y."""
        phis = self.A_T(None, y)
        ms, vpi = self.Kt_pinvT_phi0(phis)
        return -self.Bt_T(ms, vpi)

    def P_apply(self, v):
        """P v = A-bar K-bar^+ B-bar v (Neumann to Dirichlet map, Sec. 3.1)."""
        out = np.zeros_like(v)
        for L in self.loc:
            bb = np.zeros((L.m, v.shape[1]))
            bb[L.m - L.nDl:] = -v[L.gdl]                         # B-bar^i v = [0;0;0;-R_f^i v]
            np.add.at(out, L.gdl, L.Abar @ (L.Kbar_pinv @ bb))
        return out

    def P_T(self, v):
        out = np.zeros_like(v)
        for L in self.loc:
            t = L.Kbar_pinv.T @ (L.Abar.T @ v[L.gdl])
            np.add.at(out, L.gdl, -t[L.m - L.nDl:])
        return out

    def W_apply(self, v):
        th = self.o.theta
        return th * self.P_T(self.P_apply(v)) + (1.0 - th) * v

    # ------------------------------------------------------------ Eq. (nn-mixed)
    def S_theta_apply(self, mu):
        """(B~^T B~ + D~^T W D~ - B~^T K~ K~^+ B~) mu."""
        ms, psi = self.Bt_apply(mu)
        BtB = self.Bt_T(ms, psi)
        cs, mpi = self.Kt_pinv(ms, psi)
        km, kpi = self.Kt_apply(cs, mpi)
        BKKB = self.Bt_T(km, kpi)
        Dm = self.Dt_apply(mu)
        return BtB + self.Dt_T(self.W_apply(Dm)) - BKKB

    def f_tilde(self):
        return [L.f for L in self.loc], self.d_pi

    def b_theta(self):
        """(B~^T - B~^T K~ K~^+) f~ + D~^T W d~."""
        fs, dpi = self.f_tilde()
        Btf = self.Bt_T(fs, dpi)
        cs, mpi = self.Kt_pinv(fs, dpi)
        km, kpi = self.Kt_apply(cs, mpi)
        BKKf = self.Bt_T(km, kpi)
        _, adl = self.A_apply(cs)
        d_tilde = -adl                                            # d~ = -A~ K~^+ f~
        return Btf - BKKf + self.Dt_T(self.W_apply(d_tilde))

    def assemble_S_theta(self, batch=512):
        n = self.n_dl
        S = np.zeros((n, n))
        for j0 in range(0, n, batch):
            j1 = min(n, j0 + batch)
            E = np.zeros((n, j1 - j0))
            E[np.arange(j0, j1), np.arange(j1 - j0)] = 1.0
            S[:, j0:j1] = self.S_theta_apply(E)
        return S

    # ------------------------------------------------------------ solves
    def solve_direct(self):
        """mu_Delta by Cholesky of the assembled S_theta (exact solution of Eq. nn-mixed)."""
        S = self.assemble_S_theta()
        b = self.b_theta()
        mu = sla.cho_solve(sla.cho_factor(S, lower=True), b)
        return mu, S, b

    def solve_cg(self, tol=None, max_iters=None):
        """Plain CG on Eq. (nn-mixed) from mu = 0, stopped on |r_k|/|b| < tol (Sec. 4)."""
        tol = self.o.tol if tol is None else tol
        max_iters = self.o.max_iters if max_iters is None else max_iters
        b = self.b_theta()
        mu = np.zeros_like(b)
        r = b.copy()
        pvec = r.copy()
        rr = (r * r).sum(0)
        bn = np.sqrt((b * b).sum(0))
        it = 0
        while it < max_iters and np.any(np.sqrt(rr) >= tol * bn):
            q = self.S_theta_apply(pvec)
            alpha = rr / (pvec * q).sum(0)
            mu += alpha * pvec
            r -= alpha * q
            rr_new = (r * r).sum(0)
            pvec = r + (rr_new / rr) * pvec
            rr = rr_new
            it += 1
        return mu, it

    def reconstruct(self, mu_dl):
        """[c; mu_Pi] = K~^+ (f~ - B~ mu_Delta), Eq. (coarse_sol_2)."""
        fs, dpi = self.f_tilde()
        ms, psi = self.Bt_apply(mu_dl)
        cs, mu_pi = self.Kt_pinv([f - m for f, m in zip(fs, ms)], dpi - psi)
        return cs, mu_pi

    def u_eval(self, cs):
        p = self.p
        Eoff = np.concatenate([[0], np.cumsum(p.n_eval)])
        out = []
        for i, (L, c) in enumerate(zip(self.loc, cs)):
            out.append(phi(L.w, L.b, p.x_eval[Eoff[i]:Eoff[i + 1]]) @ c)
        return np.concatenate(out)

    def true_residual(self, mu):
        b = self.b_theta()
        r = b - self.S_theta_apply(mu)
        return np.sqrt((r * r).sum(0)) / np.sqrt((b * b).sum(0))


def solve(prob, opts=None, method="direct"):
    """Full oracle solve: returns dict with mu_Delta, mu_Pi, c, u_eval, iterations."""
    o = DDELMOracle(prob, opts)
    if method == "direct":
        mu, _, _ = o.solve_direct()
        it = 0
    else:
        mu, it = o.solve_cg()
    cs, mu_pi = o.reconstruct(mu)
    return dict(mu_delta=mu, mu_pi=mu_pi, c=cs, u_eval=o.u_eval(cs), iters=it, oracle=o)
