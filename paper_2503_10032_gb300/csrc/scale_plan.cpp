// Host plan of the scale gradient dL/ds (w = s w_hat, b = s b_hat, Sec. 2.2):
// buffers, GEMM phases and dot products of the reverse pass that ddelm_backward
// runs when a scale output is requested.
//
// After the adjoint solve, the persistent kernel leaves a bank of interface
// vectors (mode 4 of the CG kernel).  Per subdomain they define low-rank
// cotangents of the stored local operators,
//   Lambda-bar = PL WL^T, Psi-bar = PP WP^T, Phi-bar = PF WF^T,
//   (K^+ E_Gamma)-bar = c-hat ell^T, and a-bar, p-bar, y-bar,
// plus the coarse blocks of D_PiPi-bar and S_Pi-bar.  With Lambda = A_m K^+ E,
// Psi = E^T K K^+ E, Phi = A-bar K-bar^+ E_Delta, y = K^+ f, p = E^T K y and the
// derivative of the ridge pseudo-inverse, N = K^T K + eps^2 I = (V V^T)^{-1},
//   d(K^+) v = N^{-1} (dK^T (v - K K^+ v) - K^T dK K^+ v - d(eps^2) K^+ v),
// every contribution takes the form sum_j a_j^T dX b_j for X one of K_c, K-bar,
// A_m, A-bar and the evaluation matrix, and d(eps^2)/ds = 2 eps_rel^2 <K, dK>/M.
// The phases below form the factors a_j, b_j with the FP64 GEMM engine and the
// products dX b_j with the s-derivatives of the matrices, which the feature
// kernels assemble into the (otherwise idle) setup scratch of the wave.
#include <algorithm>
#include <cstring>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

long long rup(long long n) { return (std::max(n, 1LL) + 31) / 32 * 32; }

}  // namespace

int build_scale(Plan &P, long long &cur) {
  auto fail = [&](const char *m) {
    P.err = m;
    return DDELM_ERR_INVALID_ARG;
  };
  const int n_sub = P.n_sub, R = P.n_rhs, W = P.wave;
  const long long nd = std::max(P.n_dl, 1), np = std::max(P.n_pi, 1);
  auto take = [&](long long n) {
    long long o = cur;
    cur += rup(n);
    return o;
  };
  // column counts of the factored cotangents (the four coarse columns are zero
  // where a subdomain has fewer cross points)
  const int JL = 4 * R + 4, JP = 2 * R + 4, JF = 2 * R, Jc = R + JL + JP, NK = 2 * Jc + 2 * R, NAG = JL + JP + R;
  P.sc_JL = JL;
  P.sc_JP = JP;
  P.sc_JF = JF;
  P.sc_Jc = Jc;
  P.sc_NK = NK;
  P.sc_NAG = NAG;
  // bank of interface vectors (written by the persistent kernel) and coarse buffers
  P.o_bank_dl = take((long long)N_SD * nd * R);
  P.o_bank_pi = take((long long)N_SP * np * R);
  const long long np2 = np * np;
  P.o_cSb = take(np2);
  P.o_cC1b = take(np2);
  P.o_cC2b = take(np2);
  P.o_cC3b = take(np2);
  P.o_cDb = take(np2);
  P.o_cDX = take(np2);
  P.o_cT1 = take(np2);
  P.o_cT3 = take(np2);
  P.o_cSPb = take(np2);

  // per-subdomain buffers, laid out inside the subdomain's wave slot
  P.scsub.assign(n_sub, ScaleSub{});
  P.ssubs = P.subs;
  auto layout = [&](int i, long long base, ScaleSub &q) {
    const SubDev &d = P.subs[i];
    const long long M = d.M, m = d.m, nG = d.nG, nDl = d.nDl, nE = d.nE;
    long long c = base;
    auto t = [&](long long n) {
      long long o = c;
      c += rup(n);
      return o;
    };
    q.Ks = t(m * M);
    q.Kbs = t(m * M);
    q.As = t(nG * M);
    q.Abs = t(nDl * M);
    q.Es = t(nE * M);
    q.dshift = c - q.Ks;
    c += q.dshift;  // the derivative block
    q.Bc = t(nG * Jc);
    q.LA = t(nG * NAG);
    q.LG = t(nG * NAG);
    q.Ac = t(M * Jc);
    q.RAG = t(M * NAG);
    q.ybar = t(M * R);
    q.VtA = t(M * Jc);
    q.RK = t(M * NK);
    q.QGB = t(M * Jc);
    q.LK = t(m * NK);
    q.T2 = t(M * R);
    q.Rt = t(M * R);
    q.Vty = t(M * R);
    q.PF = t(nDl * JF);
    q.WFm = t(nDl * JF);
    q.t1 = t(M * JF);
    q.t2 = t(M * JF);
    q.t3 = t(M * JF);
    q.t4 = t(M * JF);
    q.RKb = t(M * 2 * JF);
    q.LKb = t(m * 2 * JF);
    q.V3QGB = t(M * Jc);
    q.V3VtA = t(M * Jc);
    q.V3Vty = t(M * R);
    q.V3Rt = t(M * R);
    q.OK = t(m * NK);
    q.OG = t(nG * NAG);
    q.OA = t(nG * NAG);
    q.OKb = t(m * 2 * JF);
    q.OAb = t(nDl * JF);
    q.OE = t(nE * R);
    return c - base;
  };
  std::vector<long long> need(W, 0);
  for (int i = 0; i < n_sub; ++i) {
    ScaleSub q;
    need[i % W] = std::max(need[i % W], layout(i, 0, q));
  }
  if ((int)P.slot_begin.size() != W) return fail("internal: scale slots");
  std::vector<long long> region(W);
  for (int k = 0; k < W; ++k)
    region[k] = need[k] <= P.slot_end[k] - P.slot_begin[k] ? P.slot_begin[k] : take(need[k]);
  for (int i = 0; i < n_sub; ++i) {
    layout(i, region[i % W], P.scsub[i]);
    const ScaleSub &q = P.scsub[i];
    SubDev &e = P.ssubs[i];
    e.oK = q.Ks;
    e.oKb = q.Kbs;
    e.oA = q.As;
    e.oAbar = q.Abs;
    e.oEval = q.Es;
    e.dshift = q.dshift;
  }
  // feature rows re-targeted at the scale buffers (same order as the setup's rows)
  P.srows = P.rows;
  for (auto &r : P.srows) {
    const SubDev &d = P.subs[r.sub];
    const SubDev &e = P.ssubs[r.sub];
    const long long M = d.M;
    auto remap = [&](long long off, long long &out) {
      if (off < 0) return true;
      const struct {
        long long from, to, n;
      } bufs[] = {{d.oK, e.oK, (long long)d.m * M},
                  {d.oKb, e.oKb, (long long)d.m * M},
                  {d.oA, e.oA, (long long)d.nG * M},
                  {d.oAbar, e.oAbar, (long long)d.nDl * M},
                  {d.oEval, e.oEval, (long long)d.nE * M}};
      for (const auto &b : bufs)
        if (off >= b.from && off < b.from + b.n) {
          out = b.to + (off - b.from);
          return true;
        }
      return false;
    };
    // (a point row's ca, cb, out2, out3 are unused)
    bool ok = remap(r.out0, r.out0) && remap(r.out1, r.out1);
    if (r.kind == ROW_DELTA)
      ok = ok && remap(r.out2, r.out2) && remap(r.out3, r.out3) && remap(r.ca, r.ca) && remap(r.cb, r.cb);
    if (r.kind == ROW_AM) {
      ok = ok && remap(r.ca, r.ca);
      for (int t = 0; t < 2; ++t) ok = ok && (r.am_e[t] == 0 || remap(r.am_f[t], r.am_f[t]));
    }
    if (!ok) return fail("internal: scale row remap");
  }
  // evaluation rows of each wave (rows after the special rows, subdomain by subdomain)
  {
    const int e0 = P.wave_row0[P.n_waves];
    P.wave_erow0.assign(P.n_waves + 1, int(P.srows.size()));
    int r = e0;
    for (int w = 0; w < P.n_waves; ++w) {
      P.wave_erow0[w] = r;
      while (r < (int)P.srows.size() && P.srows[r].sub < (w + 1) * W) ++r;
    }
    P.wave_erow0[P.n_waves] = int(P.srows.size());
  }

  // ---- GEMM phases (FP64 engine)
  auto begin = [&](int tile) {
    GemmPhase ph;
    ph.desc0 = int(P.gdesc.size());
    ph.tile0 = int(P.gtile.size());
    ph.ndesc = ph.ntile = 0;
    ph.skinny = 0;
    ph.tile = tile;
    return ph;
  };
  // C = alpha op(A) op(B) + beta C, C [mm x nn], k = kk
  auto add = [&](GemmPhase &ph, long long a, long long b, long long c, int mm, int nn, int kk, int lda, int ldb,
                 int ldc, int ta, int tb, double alpha, double beta) {
    if (mm <= 0 || nn <= 0) return;
    GemmDesc d;
    std::memset(&d, 0, sizeof(d));
    d.a = a;
    d.b = b;
    d.c = c;
    d.m = mm;
    d.n = nn;
    d.k = kk;
    d.lda = lda;
    d.ldb = ldb;
    d.ldc = ldc;
    d.ta = ta;
    d.tb = tb;
    d.alpha = alpha;
    d.beta = beta;
    const int di = int(P.gdesc.size());
    P.gdesc.push_back(d);
    P.gemm_flops.push_back(2.0 * mm * (double)nn * kk);
    ph.ndesc++;
    const int T = ph.tile;
    for (int x = 0; x < (mm + T - 1) / T; ++x)
      for (int y = 0; y < (nn + T - 1) / T; ++y) {
        P.gtile.push_back({di, x, y, 0});
        ph.ntile++;
      }
  };
  // coarse chain: X-bar = Sinv-bar + C1-bar D + D^T C3-bar - D^T C2-bar D (into cSb),
  // D-bar = C1-bar^T X + C3-bar X - (C2-bar + C2-bar^T) D X, S-bar = -X X-bar X,
  // D-bar += D (S-bar + S-bar^T)  (X = S_Pi^{-1}, C1 = X D^T, C2 = I - D X D^T, C3 = D X)
  P.sc_coarse.clear();
  if (P.n_pi > 0) {
    const int n = P.n_pi, ct = n <= 192 ? 16 : 64;
    const long long X = P.o_Sinv, D = P.o_Dpp;
    GemmPhase a = begin(ct);
    add(a, P.o_cC1b, D, P.o_cSb, n, n, n, n, n, n, 0, 0, 1.0, 1.0);
    add(a, D, X, P.o_cDX, n, n, n, n, n, n, 0, 0, 1.0, 0.0);
    add(a, P.o_cC2b, D, P.o_cT1, n, n, n, n, n, n, 0, 0, 1.0, 0.0);
    P.sc_coarse.push_back(a);
    GemmPhase b = begin(ct);
    add(b, D, P.o_cC3b, P.o_cSb, n, n, n, n, n, n, 1, 0, 1.0, 1.0);
    add(b, P.o_cC1b, X, P.o_cDb, n, n, n, n, n, n, 1, 0, 1.0, 0.0);
    P.sc_coarse.push_back(b);
    GemmPhase c = begin(ct);
    add(c, D, P.o_cT1, P.o_cSb, n, n, n, n, n, n, 1, 0, -1.0, 1.0);
    add(c, P.o_cC3b, X, P.o_cDb, n, n, n, n, n, n, 0, 0, 1.0, 1.0);
    P.sc_coarse.push_back(c);
    GemmPhase e = begin(ct);
    add(e, P.o_cC2b, P.o_cDX, P.o_cDb, n, n, n, n, n, n, 0, 0, -1.0, 1.0);
    add(e, X, P.o_cSb, P.o_cT3, n, n, n, n, n, n, 0, 0, 1.0, 0.0);
    P.sc_coarse.push_back(e);
    GemmPhase f = begin(ct);
    add(f, P.o_cC2b, P.o_cDX, P.o_cDb, n, n, n, n, n, n, 1, 0, -1.0, 1.0);
    add(f, P.o_cT3, X, P.o_cSPb, n, n, n, n, n, n, 0, 0, -1.0, 0.0);
    P.sc_coarse.push_back(f);
    GemmPhase g = begin(ct);
    add(g, D, P.o_cSPb, P.o_cDb, n, n, n, n, n, n, 0, 0, 1.0, 1.0);
    P.sc_coarse.push_back(g);
    GemmPhase h = begin(ct);
    add(h, D, P.o_cSPb, P.o_cDb, n, n, n, n, n, n, 0, 1, 1.0, 1.0);
    P.sc_coarse.push_back(h);
  }

  // per wave: the products of the factored cotangents
  P.sc_wave.assign(P.n_waves, {});
  P.dots.clear();
  P.wave_dot0.assign(P.n_waves + 1, 0);
  for (int w = 0; w < P.n_waves; ++w) {
    const int w0 = w * W, w1 = std::min(n_sub, w0 + W);
    auto &phs = P.sc_wave[w];
    // 1: KW = K^+E [WL WP] ; Ac[, R:R+JL] = A_m^T PL ; Ac[, R+JL:] = K_Gamma^T PP ; y-bar += A_m^T a-bar ;
    //    KpB = K^+E Bc ; QGB = Q_Gamma^T Bc ; T2 = Q2[data rows]^T f ; t1 = K-bar_Delta^T WF ; t2 = A-bar^T PF
    GemmPhase p1 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      const long long M = d.M;
      const long long KG = q.Ks + (long long)(d.m - d.nG) * M, AbarK = q.Ks + (long long)(d.m - d.nDl) * M;
      const long long KbD = q.Kbs + (long long)(d.m - d.nDl) * M;
      add(p1, d.oKpE, q.Bc + R, q.RAG, d.M, JL + JP, d.nG, d.nG, Jc, NAG, 0, 0, 1.0, 0.0);
      add(p1, d.oA, q.LA, q.Ac + R, d.M, JL, d.nG, d.M, NAG, Jc, 1, 0, 1.0, 0.0);
      add(p1, KG, q.LG + JL, q.Ac + R + JL, d.M, JP, d.nG, d.M, NAG, Jc, 1, 0, 1.0, 0.0);
      add(p1, d.oA, q.LA + JL + JP, q.ybar, d.M, R, d.nG, d.M, NAG, R, 1, 0, 1.0, 1.0);
      add(p1, d.oKpE, q.Bc, q.RK + Jc, d.M, Jc, d.nG, d.nG, Jc, NK, 0, 0, 1.0, 0.0);
      add(p1, d.oQG, q.Bc, q.QGB, d.M, Jc, d.nG, d.M, Jc, Jc, 1, 0, 1.0, 0.0);
      add(p1, d.oX, d.oF, q.T2, d.M, R, d.nI + d.nB, d.M, R, R, 1, 0, 1.0, 0.0);
      add(p1, KbD, q.WFm, q.t1, d.M, JF, d.nDl, d.M, JF, JF, 1, 0, 1.0, 0.0);
      add(p1, AbarK, q.PF, q.t2, d.M, JF, d.nDl, d.M, JF, JF, 1, 0, 1.0, 0.0);
    }
    phs.push_back(p1);
    // 2: y-bar += K_Gamma^T p-bar ; VtA = V^T Ac ; V3QGB = V3 QGB ; Rt = V3^T T2 ; t3 = V-bar^T t1 ; t4 = V-bar^T t2
    GemmPhase p2 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      const long long KG = q.Ks + (long long)(d.m - d.nG) * d.M;
      add(p2, KG, q.LG + JL + JP, q.ybar, d.M, R, d.nG, d.M, NAG, R, 1, 0, 1.0, 1.0);
      add(p2, d.oV, q.Ac, q.VtA, d.M, Jc, d.M, d.M, Jc, Jc, 1, 0, 1.0, 0.0);
      add(p2, d.oV3, q.QGB, q.V3QGB, d.M, Jc, d.M, d.M, Jc, Jc, 0, 0, 1.0, 0.0);
      add(p2, d.oV3, q.T2, q.Rt, d.M, R, d.M, d.M, R, R, 1, 0, 1.0, 0.0);
      add(p2, d.oVb, q.t1, q.t3, d.M, JF, d.M, d.M, JF, JF, 1, 0, 1.0, 0.0);
      add(p2, d.oVb, q.t2, q.t4, d.M, JF, d.M, d.M, JF, JF, 1, 0, 1.0, 0.0);
    }
    phs.push_back(p2);
    // 3: Zc = V VtA ; V3VtA = V3 VtA ; Uc = E_Gamma Bc - Q V3QGB ; Vty = V^T y-bar ; V3Rt = V3 Rt ;
    //    KbW = V-bar t3 ; Zb = V-bar t4
    GemmPhase p3 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      add(p3, d.oV, q.VtA, q.RK, d.M, Jc, d.M, d.M, Jc, NK, 0, 0, 1.0, 0.0);
      add(p3, d.oV3, q.VtA, q.V3VtA, d.M, Jc, d.M, d.M, Jc, Jc, 0, 0, 1.0, 0.0);
      add(p3, d.oX, q.V3QGB, q.LK, d.m, Jc, d.M, d.M, Jc, NK, 0, 0, -1.0, 1.0);
      add(p3, d.oV, q.ybar, q.Vty, d.M, R, d.M, d.M, R, R, 1, 0, 1.0, 0.0);
      add(p3, d.oV3, q.Rt, q.V3Rt, d.M, R, d.M, d.M, R, R, 0, 0, 1.0, 0.0);
      add(p3, d.oVb, q.t3, q.RKb + JF, d.M, JF, d.M, d.M, JF, 2 * JF, 0, 0, 1.0, 0.0);
      add(p3, d.oVb, q.t4, q.RKb, d.M, JF, d.M, d.M, JF, 2 * JF, 0, 0, 1.0, 0.0);
    }
    phs.push_back(p3);
    // 4: -QVA = -Q V3VtA ; zf = V Vty ; V3Vty = V3 Vty ; fr = f - Q V3Rt ; Ub = E_Delta WF - K-bar KbW ;
    //    -K-bar Zb
    GemmPhase p4 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      add(p4, d.oX, q.V3VtA, q.LK + Jc, d.m, Jc, d.M, d.M, Jc, NK, 0, 0, -1.0, 0.0);
      add(p4, d.oV, q.Vty, q.RK + 2 * Jc, d.M, R, d.M, d.M, R, NK, 0, 0, 1.0, 0.0);
      add(p4, d.oV3, q.Vty, q.V3Vty, d.M, R, d.M, d.M, R, R, 0, 0, 1.0, 0.0);
      add(p4, d.oX, q.V3Rt, q.LK + 2 * Jc, d.m, R, d.M, d.M, R, NK, 0, 0, -1.0, 1.0);
      add(p4, q.Kbs, q.RKb + JF, q.LKb, d.m, JF, d.M, d.M, 2 * JF, 2 * JF, 0, 0, -1.0, 1.0);
      add(p4, q.Kbs, q.RKb, q.LKb + JF, d.m, JF, d.M, d.M, 2 * JF, 2 * JF, 0, 0, -1.0, 0.0);
    }
    phs.push_back(p4);
    // 5: -QVy = -Q V3Vty
    GemmPhase p5 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      add(p5, d.oX, q.V3Vty, q.LK + 2 * Jc + R, d.m, R, d.M, d.M, R, NK, 0, 0, -1.0, 0.0);
    }
    phs.push_back(p5);
    // 6: the s-derivatives of the matrices times the right factors
    GemmPhase p6 = begin(64);
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      const long long M = d.M, sh = q.dshift;
      const long long dKG = q.Ks + sh + (long long)(d.m - d.nG) * M, dAbar = q.Ks + sh + (long long)(d.m - d.nDl) * M;
      add(p6, q.Ks + sh, q.RK, q.OK, d.m, NK, d.M, d.M, NK, NK, 0, 0, 1.0, 0.0);
      add(p6, dKG, q.RAG, q.OG, d.nG, NAG, d.M, d.M, NAG, NAG, 0, 0, 1.0, 0.0);
      add(p6, q.As + sh, q.RAG, q.OA, d.nG, NAG, d.M, d.M, NAG, NAG, 0, 0, 1.0, 0.0);
      add(p6, q.Kbs + sh, q.RKb, q.OKb, d.m, 2 * JF, d.M, d.M, 2 * JF, 2 * JF, 0, 0, 1.0, 0.0);
      add(p6, dAbar, q.RKb + JF, q.OAb, d.nDl, JF, d.M, d.M, 2 * JF, JF, 0, 0, 1.0, 0.0);
      add(p6, q.Es + sh, P.o_cout + d.w_off * R, q.OE, d.nE, R, d.M, d.M, R, R, 0, 0, 1.0, 0.0);
    }
    phs.push_back(p6);
    // dot products: the contraction terms, then the two ridge terms
    P.wave_dot0[w] = int(P.dots.size());
    for (int i = w0; i < w1; ++i) {
      const SubDev &d = P.subs[i];
      const ScaleSub &q = P.scsub[i];
      const int M = d.M;
      auto dot = [&](long long a, long long b, int rows, int cols, int lda, int ldb, int role, double coef) {
        if (rows <= 0 || cols <= 0) return;
        P.dots.push_back(DotDesc{a, b, rows, cols, lda, ldb, i, role, coef});
      };
      dot(q.LK, q.OK, d.m, NK, NK, NK, DOT_LIN, 1.0);
      dot(q.LA, q.OA, d.nG, NAG, NAG, NAG, DOT_LIN, 1.0);
      dot(q.LG, q.OG, d.nG, NAG, NAG, NAG, DOT_LIN, 1.0);
      dot(q.LKb, q.OKb, d.m, 2 * JF, 2 * JF, 2 * JF, DOT_LIN, 1.0);
      dot(q.PF, q.OAb, d.nDl, JF, JF, JF, DOT_LIN, 1.0);
      dot(d.oU, q.OE, d.nE, R, R, R, DOT_LIN, 1.0);
      dot(q.RK, q.RK + Jc, M, Jc, NK, NK, DOT_E2K, -1.0);
      dot(q.RK + 2 * Jc, q.RK + 2 * Jc + R, M, R, NK, NK, DOT_E2K, -1.0);
      dot(q.Ks, q.Ks + q.dshift, d.m, M, M, M, DOT_KDK, 1.0);
      dot(q.RKb, q.RKb + JF, M, JF, 2 * JF, 2 * JF, DOT_E2KB, -1.0);
      dot(q.Kbs, q.Kbs + q.dshift, d.m, M, M, M, DOT_KBDKB, 1.0);
    }
  }
  P.wave_dot0[P.n_waves] = int(P.dots.size());
  P.o_gs = take((long long)P.dots.size() + n_sub + 8);
  return DDELM_OK;
}

}  // namespace ddelm
