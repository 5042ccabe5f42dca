"""Brute-force dense DDELM-NN for tiny problems (test infrastructure only).

Every global matrix is formed literally and every pseudo-inverse is numpy's
``pinv``: Eq. (ddelm) gives K, B, A, f; Sec. 3 gives the partition into Pi and
Delta, D_ab, d_a, K~, B~, A~, f~, D~, d~; Sec. 3.1 gives K-bar, B-bar,
A-bar and P; Eq. (nn-mixed) and Eq. (coarse_sol_2) give the solution.  The
ridge reading of the local least-squares problems is realised literally as
rows eps_i * I appended to every K^i (zero data, zero B rows).

Only the local row blocks (features, layout) are shared with the structured
oracle; none of its algebra is.
"""
from __future__ import annotations

import numpy as np


def _blockdiag(blocks):
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    out = np.zeros((rows, cols))
    r = c = 0
    for b in blocks:
        out[r:r + b.shape[0], c:c + b.shape[1]] = b
        r += b.shape[0]
        c += b.shape[1]
    return out


def global_system(orc):
    """K, B, A, f of Eq. (ddelm) (ridge rows appended) and K-bar, B-bar, A-bar."""
    loc = orc.loc
    n_pi, n_dl = orc.n_pi, orc.n_dl
    nG = n_pi + n_dl
    Kb, Bb, fb, Kbb, Bbb = [], [], [], [], []
    A = np.zeros((nG, sum(L.K.shape[1] for L in loc)))
    Abar = np.zeros((n_dl, A.shape[1]))
    col = 0
    for L in loc:
        M = L.K.shape[1]
        Kb.append(np.vstack([L.K, np.sqrt(L.eps2) * np.eye(M)]))
        R = np.zeros((L.nG, nG))                       # R^i: Gamma -> Gamma^i
        R[np.arange(L.nPi), L.gpi] = 1.0
        R[L.nPi + np.arange(L.nDl), n_pi + L.gdl] = 1.0
        B = np.zeros((L.m + M, nG))
        B[L.m - L.nG:L.m] = -R                         # B^i = [0; 0; -R^i; 0]
        Bb.append(B)
        fb.append(np.vstack([L.f, np.zeros((M, L.f.shape[1]))]))
        A[:, col:col + M] = R.T @ L.Ahat               # A^i = F phi^i(x_Gamma) on Gamma^i
        # Sec. 3.1: K-bar^i, B-bar^i = [0;0;0;-R_f^i], A-bar^i
        Kbb.append(np.vstack([L.Kbar, np.sqrt(L.eps2_bar) * np.eye(M)]))
        Rf = np.zeros((L.nDl, n_dl))
        Rf[np.arange(L.nDl), L.gdl] = 1.0
        Bbar = np.zeros((L.m + M, n_dl))
        Bbar[L.m - L.nDl:L.m] = -Rf
        Bbb.append(Bbar)
        Abar[:, col:col + M] = Rf.T @ L.Abar
        col += M
    return dict(K=_blockdiag(Kb), B=np.vstack(Bb), A=A, f=np.vstack(fb),
                Kbar=_blockdiag(Kbb), Bbar=np.vstack(Bbb), Abar=Abar)


def solve_dense(orc, theta=None):
    """mu_Delta, mu_Pi, c from the literal global formulas."""
    th = orc.o.theta if theta is None else theta
    g = global_system(orc)
    K, B, A, f = g["K"], g["B"], g["A"], g["f"]
    n_pi = orc.n_pi
    B_pi, B_dl = B[:, :n_pi], B[:, n_pi:]
    A_pi, A_dl = A[:n_pi], A[n_pi:]
    Kp = np.linalg.pinv(K)
    D_pp = -A_pi @ Kp @ B_pi
    D_pd = -A_pi @ Kp @ B_dl
    d_p = -A_pi @ Kp @ f
    nc = K.shape[1]
    Kt = np.block([[K, B_pi], [np.zeros((n_pi, nc)), D_pp]])
    Bt = np.vstack([B_dl, D_pd])
    At = np.hstack([A_dl, np.zeros((A_dl.shape[0], n_pi))])
    ft = np.vstack([f, d_p])
    Ktp = np.linalg.pinv(Kt)
    Dt = -At @ Ktp @ Bt
    dt = -At @ Ktp @ ft
    P = g["Abar"] @ np.linalg.pinv(g["Kbar"]) @ g["Bbar"]
    W = th * P.T @ P + (1.0 - th) * np.eye(P.shape[0])
    KK = Kt @ Ktp
    S = Bt.T @ Bt + Dt.T @ W @ Dt - Bt.T @ KK @ Bt
    b = (Bt.T - Bt.T @ KK) @ ft + Dt.T @ W @ dt
    mu = np.linalg.solve(S, b)
    sol = Ktp @ (ft - Bt @ mu)
    c_all, mu_pi = sol[:nc], sol[nc:]
    cs, off = [], 0
    for L in orc.loc:
        M = L.K.shape[1]
        cs.append(c_all[off:off + M])
        off += M
    return dict(mu_delta=mu, mu_pi=mu_pi, c=cs, S=S, b=b, Kt=Kt, Bt=Bt, Dt=Dt, dt=dt,
                ft=ft, W=W, P=P)
