// Host-side plan of a DDELM-NN handle: the decomposition (points, the split
// Gamma = Pi u Delta of Sec. 3, the change of variables T^i and the modified
// flux rows A_m^i of Sec. 3.2), the index maps R^i, the workspace layout and
// the tables of every batched GEMM / Cholesky phase of the setup.
//
// The geometry follows the conventions documented in include/ddelm.h.  Every
// table is position independent (offsets, not pointers), so the whole plan is
// uploaded into the caller's workspace with one copy.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

struct V2 {
  double x, y;
};

struct EdgeRef {
  int id;
  int sv[2], ev[2];  // start / end vertex (vx, vy)
  double n[2];       // outward normal of the subdomain
};

struct Geo {
  int nx, ny;
  double x0, x1, y0, y1, hx, hy;
  const int *edge_pts;
  int H() const { return nx * (ny + 1); }
  int n_edges() const { return H() + (nx + 1) * ny; }
  bool edge_on_boundary(int eid) const {
    if (eid < H()) {
      int vy = eid / nx;
      return vy == 0 || vy == ny;
    }
    int vx = (eid - H()) / ny;
    return vx == 0 || vx == nx;
  }
  bool is_cross(const int v[2]) const { return v[0] > 0 && v[0] < nx && v[1] > 0 && v[1] < ny; }
  int pi_index(const int v[2]) const { return (v[1] - 1) * (nx - 1) + (v[0] - 1); }
  V2 vxy(const int v[2]) const { return {x0 + v[0] * hx, y0 + v[1] * hy}; }
  V2 edge_point(const EdgeRef &e, int k) const {  // k = 1..n
    int n = edge_pts[e.id];
    V2 a = vxy(e.sv), b = vxy(e.ev);
    double f = double(k) / double(n + 1);
    return {a.x + f * (b.x - a.x), a.y + f * (b.y - a.y)};
  }
};

}  // namespace

int build_plan(const ddelm_problem *prob, Plan &P) {
  if (!prob) return DDELM_ERR_INVALID_ARG;
  const ddelm_problem &pr = *prob;
  auto fail = [&](const char *m) {
    P.err = m;
    return DDELM_ERR_INVALID_ARG;
  };
  if (pr.nx < 1 || pr.ny < 1 || (long long)pr.nx * pr.ny > 65535) return fail("bad nx/ny");
  if (!(pr.x1 > pr.x0) || !(pr.y1 > pr.y0)) return fail("bad rectangle");
  if (pr.n_rhs < 1 || pr.n_rhs > 16) return fail("n_rhs must be in 1..16");
  if (pr.op != DDELM_OP_POISSON && pr.op != DDELM_OP_DIFFUSION && pr.op != DDELM_OP_BIHARMONIC)
    return fail("bad op");
  if (!pr.M || !pr.w_hat || !pr.b_hat || !pr.n_int || !pr.edge_pts) return fail("null input");
  if (pr.op == DDELM_OP_DIFFUSION && (!pr.a_int || !pr.grad_a_int)) return fail("diffusion needs a");
  const ddelm_options &o = pr.opt;
  if (!(o.theta >= 0.0 && o.theta <= 1.0)) return fail("theta must be in [0,1]");
  if (!(o.eps_rel >= 0.0) || !(o.tol > 0.0) || o.max_iters < 1) return fail("bad options");
  if (o.precision != DDELM_PREC_FP64 && o.precision != DDELM_PREC_MIXED) return fail("bad precision");
  if (o.setup_scheme < DDELM_SCHEME_AUTO || o.setup_scheme > DDELM_SCHEME_CQR2_SERIES_DW || o.setup_passes < 0 ||
      o.setup_passes > 8)
    return fail("bad setup scheme");
  if (o.barrier_timeout_ms < 0 || o.inject_barrier_stall < 0 || o.inject_barrier_stall > 1)
    return fail("bad barrier options");
  if (o.plain_flux_corners < 0 || o.plain_flux_corners > 1) return fail("bad plain_flux_corners");
  if (o.vanilla < 0 || o.vanilla > 1) return fail("bad vanilla");
  if (o.autotune < 0 || o.autotune > 1) return fail("bad autotune");
  if (o.tc_tiles < 0 || o.tc_tiles > 3) return fail("bad tc_tiles");
  if (o.trim_levels < 0 || o.trim_levels > 6) return fail("bad trim_levels");
  if (o.chol_blocked < 0 || o.chol_blocked > 1) return fail("bad chol_blocked");
  if (o.vanilla && o.theta != 0.0) return fail("vanilla DDELM takes theta = 0");
  P.opt = o;
  P.keep = o.keep_matrices != 0;
  P.inv_scale = pr.scale != 0.0 ? 1.0 / pr.scale : 0.0;
  if (pr.op == DDELM_OP_BIHARMONIC) {
    // the reweighting of the loss terms: every derivative of order k times H^k
    const double H = std::sqrt((pr.x1 - pr.x0) / pr.nx * ((pr.y1 - pr.y0) / pr.ny));
    P.w_f0 = H;
    P.w_c1 = H * H;
    P.w_f1 = H * H * H;
    P.w_int = P.w_c1 * P.w_c1;
  }
  const int nx = pr.nx, ny = pr.ny, n_sub = nx * ny;
  Geo g{nx, ny, pr.x0, pr.x1, pr.y0, pr.y1, (pr.x1 - pr.x0) / nx, (pr.y1 - pr.y0) / ny, pr.edge_pts};
  const int n_edges = g.n_edges();
  for (int e = 0; e < n_edges; ++e)
    if (pr.edge_pts[e] < 0 || pr.edge_pts[e] > 100000) return fail("bad edge_pts");
  long long sumM = 0, sumI = 0, sumE = 0;
  for (int i = 0; i < n_sub; ++i) {
    if (pr.M[i] < 1 || pr.M[i] > 1024) return fail("M must be in 1..1024");
    if (pr.n_int[i] < 0) return fail("bad n_int");
    if (pr.n_eval && pr.n_eval[i] < 0) return fail("bad n_eval");
    sumM += pr.M[i];
    sumI += pr.n_int[i];
    sumE += pr.n_eval ? pr.n_eval[i] : 0;
  }
  if (sumI > 0 && !pr.x_int) return fail("null x_int");
  if (sumE > 0 && !pr.x_eval) return fail("null x_eval");
  const int R = pr.n_rhs;
  P.n_sub = n_sub;
  P.n_rhs = R;
  P.op = pr.op;

  // ---- global Dirichlet list and Gamma numbering
  std::vector<int> bnd_off(n_edges, -1), dl_off(n_edges, -1);
  int nb = 0;
  for (int e = 0; e < n_edges; ++e)
    if (g.edge_on_boundary(e)) {
      bnd_off[e] = nb;
      nb += pr.edge_pts[e];
    }
  std::vector<int> vtx_bnd((nx + 1) * (ny + 1), -1);
  for (int vy = 0; vy <= ny; ++vy)
    for (int vx = 0; vx <= nx; ++vx)
      if (vx == 0 || vx == nx || vy == 0 || vy == ny) vtx_bnd[vy * (nx + 1) + vx] = nb++;
  // vanilla DDELM (Sec. 2.2.1, no coarse space): Pi is empty and the cross
  // points open the Delta list (in cross-point order), each shared by four subdomains
  const bool vanilla = o.vanilla != 0;
  const int n_cross = (nx - 1) * (ny - 1);
  int n_pi = vanilla ? 0 : n_cross;
  int nd = vanilla ? n_cross : 0;
  for (int e = 0; e < n_edges; ++e)
    if (!g.edge_on_boundary(e)) {
      dl_off[e] = nd;
      nd += pr.edge_pts[e];
    }
  P.n_pi = n_pi;
  P.n_dl = nd;
  P.sz.n_sub = n_sub;
  P.sz.n_edges = n_edges;
  P.sz.n_bnd = nb;
  P.sz.n_pi = n_pi;
  P.sz.n_delta = nd;
  P.sz.sum_M = sumM;
  P.sz.sum_int = sumI;
  P.sz.sum_eval = sumE;

  // ---- per-subdomain geometry
  struct SubGeo {
    std::vector<V2> bxy;
    std::vector<int> bg;
    std::vector<V2> pxy;
    std::vector<int> pg;
    std::vector<std::pair<int, int>> pv;  // vertices of the local Pi points
    std::vector<V2> dxy, dnrm;
    std::vector<int> dg;
    std::vector<double> al, be;
    std::vector<int> alp, bep;
    std::vector<std::vector<EdgeRef>> am_edges;  // per local Pi: the two edges meeting it
    std::map<int, int> dstart;                    // edge id -> index of its first Delta point
    // interface / boundary component of every point (biharmonic: 0 u, 1 Lap u)
    std::vector<int> bcomp, pcomp, dcomp;
    int np0 = 0, nd0 = 0;                         // Pi and Delta points of component 0
  };
  std::vector<SubGeo> sg(n_sub);
  const int H = g.H();
  for (int i = 0; i < n_sub; ++i) {
    const int ix = i % nx, iy = i / nx;
    int BL[2] = {ix, iy}, BR[2] = {ix + 1, iy}, TL[2] = {ix, iy + 1}, TR[2] = {ix + 1, iy + 1};
    EdgeRef edges[4] = {
        {iy * nx + ix, {BL[0], BL[1]}, {BR[0], BR[1]}, {0.0, -1.0}},
        {(iy + 1) * nx + ix, {TL[0], TL[1]}, {TR[0], TR[1]}, {0.0, 1.0}},
        {H + ix * ny + iy, {BL[0], BL[1]}, {TL[0], TL[1]}, {-1.0, 0.0}},
        {H + (ix + 1) * ny + iy, {BR[0], BR[1]}, {TR[0], TR[1]}, {1.0, 0.0}},
    };
    SubGeo &s = sg[i];
    for (auto &e : edges)
      if (g.edge_on_boundary(e.id))
        for (int k = 1; k <= pr.edge_pts[e.id]; ++k) {
          s.bxy.push_back(g.edge_point(e, k));
          s.bg.push_back(bnd_off[e.id] + k - 1);
        }
    const int *verts[4] = {BL, BR, TL, TR};
    for (auto v : verts)
      if (!g.is_cross(v) && (v[0] == 0 || v[0] == nx || v[1] == 0 || v[1] == ny)) {
        s.bxy.push_back(g.vxy(v));
        s.bg.push_back(vtx_bnd[v[1] * (nx + 1) + v[0]]);
      }
    std::map<std::pair<int, int>, int> locpi;
    for (auto v : verts)
      if (g.is_cross(v) && vanilla) {
        // an interface point of the Delta set; its flux row is the plain one of
        // Eq. (ddelm) with the corner normal resolved as the sum of the outward
        // normals of the two edges of this subdomain that meet there
        V2 nsum{0.0, 0.0};
        for (auto &e : edges)
          if ((e.sv[0] == v[0] && e.sv[1] == v[1]) || (e.ev[0] == v[0] && e.ev[1] == v[1])) {
            nsum.x += e.n[0];
            nsum.y += e.n[1];
          }
        s.dxy.push_back(g.vxy(v));
        s.dnrm.push_back(nsum);
        s.dg.push_back(g.pi_index(v));
        s.al.push_back(0.0);
        s.alp.push_back(-1);
        s.be.push_back(0.0);
        s.bep.push_back(-1);
      } else if (g.is_cross(v)) {
        locpi[{v[0], v[1]}] = int(s.pxy.size());
        s.pxy.push_back(g.vxy(v));
        s.pg.push_back(g.pi_index(v));
        s.pv.push_back({v[0], v[1]});
      }
    for (auto &e : edges) {
      if (g.edge_on_boundary(e.id)) continue;
      const int n = pr.edge_pts[e.id];
      auto a = locpi.find({e.sv[0], e.sv[1]});
      auto b = locpi.find({e.ev[0], e.ev[1]});
      s.dstart[e.id] = int(s.dxy.size());
      for (int k = 1; k <= n; ++k) {
        double f = double(k) / double(n + 1);
        s.dxy.push_back(g.edge_point(e, k));
        s.dnrm.push_back({e.n[0], e.n[1]});
        s.dg.push_back(dl_off[e.id] + k - 1);
        s.al.push_back(a != locpi.end() ? 1.0 - f : 0.0);
        s.alp.push_back(a != locpi.end() ? a->second : -1);
        s.be.push_back(b != locpi.end() ? f : 0.0);
        s.bep.push_back(b != locpi.end() ? b->second : -1);
      }
    }
    s.am_edges.resize(s.pv.size());
    for (size_t k = 0; k < s.pv.size(); ++k)
      for (auto &e : edges) {
        bool at_s = e.sv[0] == s.pv[k].first && e.sv[1] == s.pv[k].second;
        bool at_e = e.ev[0] == s.pv[k].first && e.ev[1] == s.pv[k].second;
        if (at_s || at_e) s.am_edges[k].push_back(e);
      }
  }

  // ---- biharmonic (the coupled system of Sec. 2.1): u and Lap u are both
  // interface unknowns, so every boundary, Pi and Delta point gets a second
  // row of component 1, numbered after all of component 0 (globally and within
  // each block of a subdomain); its change of variables refers to the
  // component-1 corner rows
  const int n_comp = pr.op == DDELM_OP_BIHARMONIC ? 2 : 1;
  P.nb0 = nb;
  for (auto &s : sg) {
    const int kb = int(s.bxy.size()), kp = int(s.pxy.size()), kd = int(s.dxy.size());
    s.np0 = kp;
    s.nd0 = kd;
    s.bcomp.assign(kb, 0);
    s.pcomp.assign(kp, 0);
    s.dcomp.assign(kd, 0);
    if (n_comp == 1) continue;
    for (int k = 0; k < kb; ++k) {
      const V2 xy = s.bxy[k];
      s.bxy.push_back(xy);
      s.bg.push_back(s.bg[k] + nb);
      s.bcomp.push_back(1);
    }
    for (int k = 0; k < kp; ++k) {
      const V2 xy = s.pxy[k];
      const std::pair<int, int> v = s.pv[k];
      const std::vector<EdgeRef> ae = s.am_edges[k];
      s.pxy.push_back(xy);
      s.pg.push_back(s.pg[k] + n_pi);
      s.pv.push_back(v);
      s.am_edges.push_back(ae);
      s.pcomp.push_back(1);
    }
    for (int k = 0; k < kd; ++k) {
      const V2 xy = s.dxy[k], nrm = s.dnrm[k];
      const double al = s.al[k], be = s.be[k];
      const int alp = s.alp[k], bep = s.bep[k];
      s.dxy.push_back(xy);
      s.dnrm.push_back(nrm);
      s.dg.push_back(s.dg[k] + nd);
      s.al.push_back(al);
      s.be.push_back(be);
      s.alp.push_back(alp >= 0 ? alp + kp : -1);
      s.bep.push_back(bep >= 0 ? bep + kp : -1);
      s.dcomp.push_back(1);
    }
  }
  if (n_comp == 2) {
    nb *= 2;
    n_pi *= 2;
    nd *= 2;
  }
  P.n_pi = n_pi;
  P.n_dl = nd;
  P.sz.n_bnd = nb;
  P.sz.n_pi = n_pi;
  P.sz.n_delta = nd;

  // ---- workspace layout
  P.subs.resize(n_sub);
  long long cur = 0;
  auto take = [&](long long n) {
    long long off = cur;
    cur += (std::max(n, 1LL) + 31) / 32 * 32;
    return off;
  };
  P.o_w = take(2 * sumM);
  P.o_b = take(sumM);
  P.o_xint = take(2 * sumI);
  P.o_aint = take(sumI);
  P.o_gaint = take(2 * sumI);
  P.o_fc = take(4 * sumM);
  P.o_exp2 = take(256);
  long long wo = 0, io = 0, eo = 0;
  int max_M = 0, sum_nG = 0;
  long long setup_scratch_begin = 0;
  // persistent per-subdomain operators first
  for (int i = 0; i < n_sub; ++i) {
    SubDev &d = P.subs[i];
    const SubGeo &s = sg[i];
    d.M = pr.M[i];
    d.nI = pr.n_int[i];
    d.nB = int(s.bxy.size());
    d.nPi = int(s.pxy.size());
    d.nDl = int(s.dxy.size());
    d.nG = d.nPi + d.nDl;
    d.m = d.nI + d.nB + d.nG;
    d.nE = pr.n_eval ? pr.n_eval[i] : 0;
    d.w_off = wo;
    d.int_off = io;
    d.eval_off = eo;
    wo += d.M;
    io += d.nI;
    eo += d.nE;
    max_M = std::max(max_M, d.M);
    d.loc_off = sum_nG;
    sum_nG += d.nG;
    const long long M = d.M, m = d.m, nG = d.nG, nDl = d.nDl;
    d.oX = take(m * M);  // the final Q of K_c (needed by every solve)
    d.oA = take(nG * M);
    d.oEval = take(d.nE * M);
    d.oV = take(M * M);
    d.oVb = take(M * M);  // R^{-1} of K-bar (kept: the scale gradient reuses it)
    d.oV3 = take(M * M);
    d.oQG = take(nG * M);
    d.oKpE = take(M * nG);
    d.oLam = take(nG * nG);
    d.oLamT = take(nG * nG);
    d.oPsi = take(nG * nG);
    d.oPhi = take(nDl * nDl);
    d.oPhiT = take(nDl * nDl);
    d.oF = take((d.nI + d.nB) * R);
    d.oT = take(M * R);
    d.oQtf = take(M * R);
    d.oY = take(M * R);
    d.oAy = take(nG * R);
    d.oP = take(nG * R);
    d.oC = take(M * R);
    d.oU = take((long long)d.nE * R);
  }
  P.max_M = max_M;
  P.sum_nG = sum_nG;
  // coarse matrices
  const long long np = std::max(n_pi, 1);
  P.o_Dpp = take(np * np);
  P.o_Spi = take(np * np);
  P.o_Vpi = take(np * np);
  P.o_Sinv = take(np * np);
  P.o_C1 = take(np * np);
  P.o_C2 = take(np * np);
  P.o_C3 = take(np * np);
  P.o_SpiR = take(np * np);
  // CG vectors: 12 Delta vectors, 14 Pi vectors, 9 local slabs, reductions
  const long long nd_ = std::max(nd, 1), nR = R;
  P.o_cg = take(12 * nd_ * nR + 14 * np * nR + 2048 * 32 + 128);
  P.o_loc = take(9LL * sum_nG * nR);
  P.o_status = take(4 * n_sub + 64);
  P.o_eps = take(2LL * n_sub);
  // solve-call staging: the caller's f, g in, c, mu, u out (fixed addresses, so
  // one captured graph serves every call)
  P.o_fin = take(sumI * R);
  P.o_gin = take((long long)nb * R);
  P.o_cout = take(sumM * R);
  P.o_muout = take((long long)(n_pi + nd) * R);
  P.o_uout = take(sumE * R);
  // MIXED: FP32 copies of the local and coarse operators and the vectors of the
  // inner FP32 CG (float offsets from the start of this region)
  if (o.precision == DDELM_PREC_MIXED) {
    for (const auto &d : P.subs)
      if (d.nG > 256) return fail("MIXED precision supports at most 256 interface points per subdomain");
    long long fcur = 0;
    auto ftake = [&](long long n) {
      long long off = fcur;
      fcur += (std::max(n, 1LL) + 63) / 64 * 64;
      return off;
    };
    for (int i = 0; i < n_sub; ++i) {
      SubDev &d = P.subs[i];
      const long long g2 = (long long)d.nG * d.nG, l2 = (long long)d.nDl * d.nDl;
      d.oLam32 = ftake(g2);
      d.oLamT32 = ftake(g2);
      d.oPsi32 = ftake(g2);
      d.oPhi32 = ftake(l2);
      d.oPhiT32 = ftake(l2);
      P.conv.push_back({d.oLam, d.oLam32, g2});
      P.conv.push_back({d.oLamT, d.oLamT32, g2});
      P.conv.push_back({d.oPsi, d.oPsi32, g2});
      P.conv.push_back({d.oPhi, d.oPhi32, l2});
      P.conv.push_back({d.oPhiT, d.oPhiT32, l2});
    }
    const long long np2 = (long long)std::max(n_pi, 1) * std::max(n_pi, 1);
    P.f_Sinv = ftake(np2);
    P.f_C1 = ftake(np2);
    P.f_C2 = ftake(np2);
    P.f_C3 = ftake(np2);
    if (n_pi > 0) {
      P.conv.push_back({P.o_Sinv, P.f_Sinv, np2});
      P.conv.push_back({P.o_C1, P.f_C1, np2});
      P.conv.push_back({P.o_C2, P.f_C2, np2});
      P.conv.push_back({P.o_C3, P.f_C3, np2});
    }
    const long long ndR = (long long)std::max(nd, 1) * R, npR = (long long)std::max(n_pi, 1) * R;
    P.f_dl = ftake(6 * ndR);
    P.f_pv = ftake(7 * npR);
    P.f_slab = ftake(8LL * sum_nG * R);
    P.n_f32 = fcur;
    P.o_f32 = take((fcur + 1) / 2);
  }
  // inspection copies
  if (P.keep) {
    P.o_keepX = cur;
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      take(2LL * d.m * d.M + (long long)d.nG * d.M);
    }
  }
  // setup scratch (not needed after setup)
  setup_scratch_begin = cur;
  // factorisation scheme of [K; eps I] (shifted CholeskyQR, Sec. 2.2 pseudo-inverses)
  {
    int sch = o.setup_scheme;
    if (sch == DDELM_SCHEME_AUTO)
      sch = o.precision != DDELM_PREC_MIXED ? DDELM_SCHEME_FP64CQR3
                                            : (max_M >= 512 ? DDELM_SCHEME_FP32 : DDELM_SCHEME_CQR2_SERIES_DW);
    P.scheme = sch;
    P.dw_auto = o.setup_scheme == DDELM_SCHEME_AUTO && sch == DDELM_SCHEME_CQR2_SERIES_DW;
    if (sch == DDELM_SCHEME_FP64CQR3) {
      P.n_pass = 2;
      P.polish = false;
      P.tri_v = true;
    } else if (sch == DDELM_SCHEME_CQR2_SERIES || sch == DDELM_SCHEME_CQR2_SERIES_DW) {
      P.n_pass = 2;
      P.polish = true;
      P.tri_v = false;
    } else {
      // cond(G + eps^2 I) <= M / eps_rel^2 (tr G <= M lambda_max is attained when
      // one direction dominates, as with tanh features); each shifted FP32 pass
      // divides the condition number by about 1/shift_rel = 1e4, and the last,
      // unshifted pass needs it near 1.
      const double eps2 = std::max(o.eps_rel * o.eps_rel, 1e-300);
      const int auto_pass = int(std::ceil(std::log10(std::max(10.0, max_M / eps2)) / 4.0));
      P.n_pass = o.setup_passes > 0 ? o.setup_passes : std::min(8, std::max(2, auto_pass));
      if (P.n_pass < 2) return fail("the FP32 scheme needs at least two shifted passes");
      P.polish = true;
      P.tri_v = false;
    }
  }
  // per variant (K, K-bar): Gram, two pass factors, two ridge blocks, two
  // accumulated products, FP32 Cholesky work, last factor and R^{-1}
  struct VarScr {
    long long G, Va, Vb, Za, Zb, Ta, Tb, W32, V3, V;
  };
  struct Scr {
    long long Kb, Y1, Y1b, Abar, QbD, AV, AbV;
    VarScr v[2];
  };
  // Setup scratch is shared by the subdomains of different waves: subdomain i
  // uses slot i % W, sized for the largest subdomain mapped to it.
  {
    const double per_sub_bytes = [&] {
      double mx = 0;
      for (const auto &d : P.subs) {
        const double mM = double(d.m) * d.M, MM = double(d.M) * d.M;
        double b = 8.0 * (3 * mM + 18 * MM + 4.0 * d.nG * d.M);
        if (o.precision == DDELM_PREC_MIXED) b += 36.0 * mM + 36.0 * MM;  // BF16 slices of one phase
        mx = std::max(mx, b);
      }
      return mx;
    }();
    const double budget = 48.0 * (1ull << 30);
    int W = o.setup_wave > 0 ? o.setup_wave : n_sub;
    if (o.setup_wave <= 0 && per_sub_bytes * n_sub > budget)
      W = std::max(1, int(budget / std::max(per_sub_bytes, 1.0)));
    W = std::min(W, n_sub);
    P.wave = W;
    P.n_waves = (n_sub + W - 1) / W;
  }
  const int W = P.wave;
  std::vector<Scr> slot(W);
  for (int k = 0; k < W; ++k) {
    long long M = 1, m = 1, nG = 1, nDl = 1;
    for (int i = k; i < n_sub; i += W) {
      const SubDev &d = P.subs[i];
      M = std::max<long long>(M, d.M);
      m = std::max<long long>(m, d.m);
      nG = std::max<long long>(nG, d.nG);
      nDl = std::max<long long>(nDl, d.nDl);
    }
    Scr &c = slot[k];
    c.Kb = take(m * M);
    c.Y1 = take(m * M);
    c.Y1b = take(m * M);
    c.Abar = take(nDl * M);
    c.QbD = take(nDl * M);
    c.AV = take(nG * M);
    c.AbV = take(nDl * M);
    for (int t = 0; t < 2; ++t) {
      VarScr &v = c.v[t];
      v.G = take(M * M);
      v.Va = take(M * M);
      v.Vb = take(M * M);
      v.Za = take(M * M);
      v.Zb = take(M * M);
      v.Ta = take(M * M);
      v.Tb = take(M * M);
      v.W32 = take(M * M);  // 2 M^2 floats
      v.V3 = t == 0 ? -1 : take(M * M);
      v.V = -1;  // R^{-1} of both variants is persistent
    }
    P.slot_begin.push_back(c.Kb);
    P.slot_end.push_back(cur);
  }
  std::vector<Scr> scr(n_sub);
  for (int i = 0; i < n_sub; ++i) {
    SubDev &d = P.subs[i];
    scr[i] = slot[i % W];
    scr[i].v[0].V3 = d.oV3;  // persistent for K
    scr[i].v[0].V = d.oV;
    d.oKb = scr[i].Kb;
    d.oY1 = scr[i].Y1;
    d.oY1b = scr[i].Y1b;
    d.oAbar = scr[i].Abar;
    scr[i].v[1].V = d.oVb;
    // the Q updates alternate between the feature buffer and the other one;
    // the features go where the last update lands in oX
    d.oK = (P.n_pass % 2 == 0) ? d.oX : d.oY1;
  }
  (void)setup_scratch_begin;

  // ---- special rows
  std::vector<int> sub_row0(n_sub + 1, 0);
  {
    size_t nr = 0;
    for (const auto &d : P.subs) nr += (size_t)d.nB + 2 * (size_t)d.nPi + d.nDl + d.nE;
    P.rows.reserve(nr);
  }
  for (int i = 0; i < n_sub; ++i) {
    sub_row0[i] = int(P.rows.size());
    const SubDev &d = P.subs[i];
    const SubGeo &s = sg[i];
    const long long M = d.M;
    auto base = [&](int kind) {
      SpecialRow r;
      std::memset(&r, 0, sizeof(r));
      r.kind = kind;
      r.sub = i;
      r.out1 = -1;
      return r;
    };
    for (int k = 0; k < d.nB; ++k) {  // boundary rows of K_c and K-bar
      SpecialRow r = base(ROW_POINT);
      r.comp = s.bcomp[k];
      r.x = s.bxy[k].x;
      r.y = s.bxy[k].y;
      r.out0 = d.oK + (long long)(d.nI + k) * M;
      r.out1 = d.oKb + (long long)(d.nI + k) * M;
      P.rows.push_back(r);
    }
    const int g0 = d.nI + d.nB;
    auto pi_row = [&](int k) { return d.oK + (long long)(g0 + k) * M; };  // phi at local Pi point k
    for (int k = 0; k < d.nPi; ++k) {  // Pi rows: point values in K_c and K-bar
      SpecialRow r = base(ROW_POINT);
      r.comp = s.pcomp[k];
      r.x = s.pxy[k].x;
      r.y = s.pxy[k].y;
      r.out0 = pi_row(k);
      r.out1 = d.oKb + (long long)(g0 + k) * M;
      P.rows.push_back(r);
    }
    for (int k = 0; k < d.nDl; ++k) {
      // K_c Delta row (also A-bar row): (T^i)^{-1} C phi, or C phi without the
      // change of variables; K-bar Delta row (also A_m Delta row): F phi
      SpecialRow r = base(ROW_DELTA);
      r.comp = s.dcomp[k];
      r.x = s.dxy[k].x;
      r.y = s.dxy[k].y;
      r.nx = s.dnrm[k].x;
      r.ny = s.dnrm[k].y;
      r.ca = r.cb = -1;
      if (o.use_change_of_vars) {
        if (s.alp[k] >= 0) {
          r.alpha = s.al[k];
          r.ca = pi_row(s.alp[k]);
        }
        if (s.bep[k] >= 0) {
          r.beta = s.be[k];
          r.cb = pi_row(s.bep[k]);
        }
      }
      r.out0 = d.oK + (long long)(g0 + d.nPi + k) * M;
      r.out1 = d.oAbar + (long long)k * M;
      r.out2 = d.oKb + (long long)(g0 + d.nPi + k) * M;
      r.out3 = d.oA + (long long)(d.nPi + k) * M;
      P.rows.push_back(r);
    }
    for (int k = 0; k < d.nPi; ++k) {  // A_m corner rows from the flux rows of the two edges
      SpecialRow a = base(ROW_AM);
      a.comp = s.pcomp[k];
      a.out0 = d.oA + (long long)k * M;
      a.ca = pi_row(a.comp ? k - s.np0 : k);  // phi at the corner (component 0's row)
      for (int t = 0; t < 2; ++t) {
        const EdgeRef &e = s.am_edges[k][t];
        a.am_n[t][0] = e.n[0];
        a.am_n[t][1] = e.n[1];
        // plain flux rows: the corner's own flux only (no edge points, weight 1)
        a.am_e[t] = o.plain_flux_corners ? 0 : pr.edge_pts[e.id];
        // an edge meeting a cross point is an interface edge: its Delta points are
        // the e points the mean runs over
        a.am_f[t] = d.oA + (long long)(d.nPi + s.dstart.at(e.id) + a.comp * s.nd0) * M;
      }
      P.rows.push_back(a);
    }
  }
  sub_row0[n_sub] = int(P.rows.size());
  P.wave_row0.resize(P.n_waves + 1);
  for (int w = 0; w < P.n_waves; ++w) P.wave_row0[w] = sub_row0[w * W];
  P.wave_row0[P.n_waves] = sub_row0[n_sub];
  // evaluation rows
  if (sumE > 0) {
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      for (int k = 0; k < d.nE; ++k) {
        SpecialRow r;
        std::memset(&r, 0, sizeof(r));
        r.kind = ROW_POINT;
        r.sub = i;
        r.out1 = -1;
        r.x = pr.x_eval[2 * (d.eval_off + k)];
        r.y = pr.x_eval[2 * (d.eval_off + k) + 1];
        r.out0 = d.oEval + (long long)k * d.M;
        P.rows.push_back(r);
      }
    }
  }

  // ---- int tables
  auto &I = P.ints;
  for (int i = 0; i < n_sub; ++i) {
    SubDev &d = P.subs[i];
    d.gpi_off = int(I.size());
    for (int v : sg[i].pg) I.push_back(v);
    d.gdl_off = int(I.size());
    for (int v : sg[i].dg) I.push_back(v);
    d.bnd_off = int(I.size());
    for (int v : sg[i].bg) I.push_back(v);
  }
  P.o_pi_own = int(I.size());
  I.resize(I.size() + 8 * (size_t)n_pi, -1);
  P.o_dl_own = int(I.size());
  I.resize(I.size() + 8 * (size_t)nd, -1);
  {
    std::vector<int> cnt(n_pi, 0), cntd(nd, 0);
    for (int i = 0; i < n_sub; ++i) {
      for (size_t k = 0; k < sg[i].pg.size(); ++k) {
        int gi = sg[i].pg[k];
        int c = cnt[gi]++;
        if (c >= 4) return fail("internal: Pi point with more than four subdomains");
        I[P.o_pi_own + 8 * gi + 2 * c] = i;
        I[P.o_pi_own + 8 * gi + 2 * c + 1] = int(k);
      }
      for (size_t k = 0; k < sg[i].dg.size(); ++k) {
        int gi = sg[i].dg[k];
        int c = cntd[gi]++;
        if (c >= 4) return fail("internal: Delta point with more than four subdomains");
        I[P.o_dl_own + 8 * gi + 2 * c] = i;
        I[P.o_dl_own + 8 * gi + 2 * c + 1] = int(k);
      }
    }
    // four owners exactly at the cross points of vanilla DDELM (the first n_cross
    // Delta points of each component)
    const int nd1 = nd / n_comp;
    for (int gd = 0; gd < nd; ++gd)
      if (cntd[gd] != ((vanilla && gd % nd1 < n_cross) ? 4 : 2))
        return fail("internal: Delta point with the wrong number of subdomains");
  }
  // per global Dirichlet point: up to 2 (sub, local boundary row) owners (adjoint scatter)
  P.o_bnd_own = int(I.size());
  I.resize(I.size() + 4 * (size_t)nb, -1);
  {
    std::vector<int> cnt(nb, 0);
    for (int i = 0; i < n_sub; ++i)
      for (size_t k = 0; k < sg[i].bg.size(); ++k) {
        const int gb = sg[i].bg[k];
        const int c = cnt[gb]++;
        if (c >= 2) return fail("internal: boundary point with more than two subdomains");
        I[P.o_bnd_own + 4 * gb + 2 * c] = i;
        I[P.o_bnd_own + 4 * gb + 2 * c + 1] = int(k);
      }
  }
  P.o_tasks_pi = int(I.size());
  for (int i = 0; i < n_sub; ++i)
    for (int k = 0; k < P.subs[i].nPi; ++k) {
      I.push_back(i);
      I.push_back(k);
    }
  P.n_tasks_pi = (int(I.size()) - P.o_tasks_pi) / 2;
  P.o_tasks_dl = int(I.size());
  for (int i = 0; i < n_sub; ++i)
    for (int k = 0; k < P.subs[i].nDl; ++k) {
      I.push_back(i);
      I.push_back(k);
    }
  P.n_tasks_dl = (int(I.size()) - P.o_tasks_dl) / 2;
  P.o_tasks_g = int(I.size());
  for (int i = 0; i < n_sub; ++i)
    for (int k = 0; k < P.subs[i].nG; ++k) {
      I.push_back(i);
      I.push_back(k);
    }
  P.n_tasks_g = (int(I.size()) - P.o_tasks_g) / 2;
  P.o_tasks_c = int(I.size());
  for (int i = 0; i < n_sub; ++i)
    for (int k = 0; k < P.subs[i].M; ++k) {
      I.push_back(i);
      I.push_back(k);
    }
  P.n_tasks_c = (int(I.size()) - P.o_tasks_c) / 2;
  // slab rows of the owners of every Delta point (4 per point, -1 past the
  // owners), by global point and by local interface row (-1 on Pi rows): the
  // gathers read slabs in one step
  while (I.size() % 4) I.push_back(-1);  // int4 reads
  P.o_dl_rows = int(I.size());
  for (int gd = 0; gd < nd; ++gd)
    for (int o = 0; o < 4; ++o) {
      const int s = I[P.o_dl_own + 8 * gd + 2 * o], l = I[P.o_dl_own + 8 * gd + 2 * o + 1];
      I.push_back(s >= 0 ? P.subs[s].loc_off + P.subs[s].nPi + l : -1);
    }
  P.o_gam_rows = int(I.size());
  I.resize(I.size() + 4 * (size_t)sum_nG, -1);
  for (int i = 0; i < n_sub; ++i) {
    const SubDev &d = P.subs[i];
    for (int b = 0; b < d.nDl; ++b) {
      const int gd = sg[i].dg[b];
      for (int o = 0; o < 4; ++o)
        I[P.o_gam_rows + 4 * (d.loc_off + d.nPi + b) + o] = I[P.o_dl_rows + 4 * gd + o];
    }
  }

  // ---- GEMM phases
  // FP64 GEMM tiles; MIXED setup phases run on the tensor-core path and need none
  bool fp64_tiles = true;
  auto phase_begin = [&](int skinny = 0, int tile = 64) {
    GemmPhase ph;
    ph.desc0 = int(P.gdesc.size());
    ph.tile0 = int(P.gtile.size());
    ph.ndesc = ph.ntile = 0;
    ph.skinny = skinny;
    ph.tile = tile;
    return ph;
  };
  auto add = [&](GemmPhase &ph, long long a, long long b, long long c, int m, int n, int k, int lda,
                 int ldb, int ldc, int ta, int tb, int flags, double alpha, double beta,
                 bool upper_tiles = false) {
    if (m <= 0 || n <= 0) return;
    GemmDesc d;
    std::memset(&d, 0, sizeof(d));
    d.a = a;
    d.b = b;
    d.c = c;
    d.m = m;
    d.n = n;
    d.k = k;
    d.lda = lda;
    d.ldb = ldb;
    d.ldc = ldc;
    d.ta = ta;
    d.tb = tb;
    d.flags = flags;
    d.syrk = upper_tiles ? 1 : 0;
    d.alpha = alpha;
    d.beta = beta;
    int di = int(P.gdesc.size());
    P.gdesc.push_back(d);
    ph.ndesc++;
    // algorithmic flops: only the products that can be nonzero
    double f = 2.0 * m * (double)n * k;
    const bool bu = (flags & GEMM_B_UPPER) && k == n, au = (flags & GEMM_A_UPPER) && k == m;
    if (bu && au) f /= 3.0;
    else if (bu || au || upper_tiles) f /= 2.0;
    P.gemm_flops.push_back(f);
    if (!fp64_tiles) return;
    if (ph.skinny) {
      for (int x = 0; x < (m + 31) / 32; ++x) {
        P.gtile.push_back({di, x, 0, 0});
        ph.ntile++;
      }
      return;
    }
    const int T = ph.tile, tm = (m + T - 1) / T, tn = (n + T - 1) / T;
    for (int x = 0; x < tm; ++x)
      for (int y = 0; y < tn; ++y) {
        if (upper_tiles && x > y) continue;
        P.gtile.push_back({di, x, y, 0});
        ph.ntile++;
      }
  };
  auto push = [&](GemmPhase &ph) { P.setup_gemm.push_back(ph); };
  // ---- the setup sequence: per wave the features, then the factorisation of
  // [K; eps I] and [K-bar; eps-bar I] by shifted CholeskyQR with every O(m M^2)
  // and O(M^3) product a GEMM phase, then the local operators.
  const bool fp32 = P.scheme == DDELM_SCHEME_FP32;
  const bool series = P.scheme == DDELM_SCHEME_CQR2_SERIES || P.scheme == DDELM_SCHEME_CQR2_SERIES_DW;
  const bool dw = P.scheme == DDELM_SCHEME_CQR2_SERIES_DW;  // double-FP32 Cholesky factors
  fp64_tiles = o.precision != DDELM_PREC_MIXED;
  // MIXED, FP64 passes: the Cholesky kernel (FP64 on CUDA cores, one SM per
  // matrix) inverts only the 128 x 128 diagonal blocks of R
  constexpr int INVB = 128;
  // MIXED, FP32 scheme, every subdomain with M >= 768 and at most 256
  // subdomains: the shifted passes (preconditioners whose Grams the shift keeps
  // at condition <= ~1e4, so the blocked factorisation's explicit-inverse
  // panels lose nothing) run as blocked FP64 passes in place, where the FP32
  // kernel's one CTA per matrix would leave most SMs idle; the last, unshifted
  // pass keeps the FP32 kernel (in its own work buffer: the polish reads the
  // Gram after it).  Measured: M = 1000 on a 4x4 grid 5.25 -> 6.30 solves/s;
  // M in 200..800 on 16x16 2.77 -> 2.63 and M = 1000 on 32x32 unchanged (the
  // block phases' tensor-core and slicing work outweighs or matches the saving).
  int min_M = 1 << 30;
  for (int i = 0; i < n_sub; ++i) min_M = std::min(min_M, P.subs[i].M);
  const bool fp32_blocked = fp32 && o.precision == DDELM_PREC_MIXED && min_M >= 768 && n_sub <= 256;
  const bool blocked_inv = o.precision == DDELM_PREC_MIXED;
  const bool blocked_fact = blocked_inv && o.chol_blocked;
  const int N = P.n_pass;
  // BF16 slice levels (MIXED): a Gram feeding a shifted Cholesky only has to be
  // accurate well below the shift; the later Grams, whose residual the series
  // must remove, keep 54 bits.  Products of the triangular factors (R^{-1}
  // accumulated pass by pass) span many orders of magnitude inside a row, and
  // the slice truncation is relative to the row maximum: they keep 60 bits.
  // The Q and ridge-block updates and the local-operator products keep 54 bits
  // as well.  Measured by removing levels one class at a time: one level fewer
  // on the updates moves the local operator Lambda by 8e-8 (8x8, M = 400),
  // beyond the ~1e-8 spread of two FP64 factorisations of the same problems;
  // one fewer on the local-operator products leaves the 8x8 case unchanged but
  // moves Phi (3e-9) and u (4e-7) of smaller test cases past their parity
  // bounds; one fewer on the later Grams fails the series check.
  const int lv_exact = 9, lv_factor = 10, lv_first64 = 6, lv_shifted32 = 5, lv_small = 4, lv_tiny = 3;
  const int lv_update = lv_exact, lv_ops = lv_exact;
  // cls: the phase's class for the level-trim experiment option (1 Grams after
  // the first pass, 2 Q and Z updates, 4 products of triangular factors,
  // 8 local operators and their inputs, 16 the first Gram; 0 the series terms)
  auto gemm_step = [&](GemmPhase &ph, int levels, int cls) {
    if (o.trim_levels > 0 && (o.trim_mask & cls)) levels = std::max(3, levels - o.trim_levels);
    P.steps.push_back({STEP_GEMM, int(P.setup_gemm.size())});
    P.setup_gemm.push_back(ph);
    P.setup_levels.push_back(levels);
  };
  auto chol_step = [&](int desc0) {
    P.steps.push_back({STEP_CHOL, int(P.chol_passes.size())});
    P.chol_passes.push_back(CholPhase{desc0, int(P.cdesc.size()) - desc0});
  };
  auto matop_step = [&](int desc0) {
    P.steps.push_back({STEP_MATOP, int(P.matop_phases.size())});
    P.matop_phases.push_back(MatopPhase{desc0, int(P.mdesc.size()) - desc0});
  };
  const int TU = P.tri_v ? GEMM_B_UPPER : 0;  // the last factor / R^{-1} as right operand
  const int TA = P.tri_v ? GEMM_A_UPPER : 0;  // ... as left operand
  for (int w = 0; w < P.n_waves; ++w) {
    const int w0 = w * W, w1 = std::min(n_sub, w0 + W);
    P.steps.push_back({STEP_FEAT, w});
    // Q_k of variant t (0: K, 1: K-bar) lives in the feature buffer for even k
    auto qk = [&](int i, int t, int k) -> long long {
      const SubDev &d = P.subs[i];
      const long long F = t == 0 ? d.oK : d.oKb;
      const long long O = t == 0 ? (d.oK == d.oX ? d.oY1 : d.oX) : d.oY1b;
      return (k % 2) ? O : F;
    };
    auto vk = [&](int i, int t, int k) { return (k % 2) ? scr[i].v[t].Vb : scr[i].v[t].Va; };  // pass-k factor
    auto zk = [&](int i, int t, int k) { return (k % 2) ? scr[i].v[t].Zb : scr[i].v[t].Za; };  // ridge block after pass k
    auto tk = [&](int i, int t, int k) { return k == 0 ? vk(i, t, 0) : (k % 2) ? scr[i].v[t].Ta : scr[i].v[t].Tb; };
    // Gram of the features.  K_c and K-bar share their interior and boundary
    // rows (Sec. 3.1 changes only the interface rows): G_common = K_IB^T K_IB
    // once, copied, then each adds the Gram of its own interface rows.
    {
      const int lv0 = fp32 && N > 0 ? lv_shifted32 : lv_first64;
      GemmPhase ph = phase_begin();
      for (int i = w0; i < w1; ++i) {
        const SubDev &d = P.subs[i];
        add(ph, qk(i, 0, 0), qk(i, 0, 0), scr[i].v[0].G, d.M, d.M, d.nI + d.nB, d.M, d.M, d.M, 1, 0, 0, 1.0, 0.0,
            true);
      }
      gemm_step(ph, lv0, 16);
      const int m0 = int(P.mdesc.size());
      for (int i = w0; i < w1; ++i)
        P.mdesc.push_back(MatopDesc{scr[i].v[0].G, 0, scr[i].v[1].G, P.subs[i].M, 3, 2 * i + 1, -1});
      matop_step(m0);  // G-bar = G_common
      GemmPhase ph2 = phase_begin();
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t) {
          const SubDev &d = P.subs[i];
          const long long rows = qk(i, t, 0) + (long long)(d.nI + d.nB) * d.M;  // the nG interface rows
          add(ph2, rows, rows, scr[i].v[t].G, d.M, d.M, d.nG, d.M, d.M, d.M, 1, 0, 0, 1.0, 1.0, true);
        }
      gemm_step(ph2, lv0, 16);
    }
    for (int k = 0; k <= N; ++k) {
      const bool last = k == N;
      if (last && series) break;  // the series replaces the last Cholesky
      // Cholesky pass k: G = Q_k^T Q_k + Z_k^T Z_k (k = 0: Y^T Y and the ridge)
      const int c0 = int(P.cdesc.size());
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t) {
          const SubDev &d = P.subs[i];
          const VarScr &v = scr[i].v[t];
          CholDesc c;
          std::memset(&c, 0, sizeof(c));
          c.g = v.G;
          c.v = (last && !P.polish) ? v.V3 : vk(i, t, k);
          c.z = k == 0 ? zk(i, t, 0) : -1;
          c.w = v.W32;
          c.M = d.M;
          c.m = d.m;
          c.ridge = k == 0;
          c.band = 0;
          c.status = 2 * i + t;
          c.eps_rel = o.eps_rel;
          if (!fp32) {
            // s = 11 ((m+M) M + M (M+1)) u tr covers FP64 rounding of the Gram; with
            // the tensor-core Gram the shift also covers its slice truncation
            const double u = 1.1102230246251565e-16;
            c.prec = 0;
            c.shift_kind = k == 0 ? 1 : 0;
            c.shift_rel = 11.0 * (double(d.m + d.M) * d.M + double(d.M) * (d.M + 1)) * u;
            if (o.precision == DDELM_PREC_MIXED)
              c.shift_rel = std::max(c.shift_rel, 4.0 * d.m * std::pow(64.0, -lv_first64));
            if (dw && k == 0) {
              P.dw_fallback.push_back({int(P.cdesc.size()), c.shift_rel});
              // double-FP32 factor of the shifted first pass: the same bound with u = 2^-46.
              // The unshifted second pass stays FP64: its factor leaves |E| ~ M u cond(G1)
              // for the series, about 4e-7 in FP64 but near the 1e-4 limit at u = 2^-46.
              c.prec = 2;
              c.shift_rel = std::max(c.shift_rel, 11.0 * (double(d.m + d.M) * d.M + double(d.M) * (d.M + 1)) *
                                                      std::ldexp(1.0, -46));
            }
          } else {
            // FP32 factor: the shift keeps the FP32 Cholesky away from breakdown and
            // limits the condition number each pass removes to about 1/shift
            // (MIXED: the shifted passes blocked in FP64, above)
            c.prec = (fp32_blocked && !last) ? 0 : 1;
            c.shift_kind = last ? 0 : 2;
            c.shift_rel = std::max(1e-4, 2.0 * d.M * 5.9604644775390625e-8);
          }
          c.epsout = -1;
          if (blocked_inv && d.M > INVB && c.prec != 1) {
            // R^{-1} beyond the diagonal blocks comes from the tensor cores below;
            // the ridge block eps R^{-1} after it
            c.inv_block = INVB;
            if (c.z >= 0) {
              c.epsout = P.o_eps + 2 * i + t;
              c.z = -1;
            }
          }
          P.cdesc.push_back(c);
        }
      // blocked factorisation (FP64 passes in MIXED, M > INVB): the diagonal
      // additions of the whole matrix, then per INVB-wide diagonal block r:
      // the FP64 kernel factors and inverts the block (R_rr, V_rr = R_rr^{-1});
      // the panel R[r, r+1:] = V_rr^T A[r, r+1:] (in place) and the trailing
      // update A[r+1:, r+1:] -= R[r, r+1:]^T R[r, r+1:] (upper tiles) are
      // tensor-core GEMMs; the back substitution below completes V = R^{-1}.
      // The FP64 pipe keeps only the diagonal blocks' work.
      const bool block_this = (blocked_fact || (fp32_blocked && !last)) && P.cdesc[c0].prec == 0;
      if (block_this) {
        int maxnb = 0;
        for (int q = c0; q < int(P.cdesc.size()); ++q) {
          CholDesc &c = P.cdesc[q];
          if (c.M > INVB) {
            c.mode = 1;
            c.inv_block = 0;
            maxnb = std::max(maxnb, (c.M + INVB - 1) / INVB);
          }
        }
        chol_step(c0);
        for (int jb = 0; jb < maxnb; ++jb) {
          const int cb0 = int(P.cdesc.size());
          for (int i = w0; i < w1; ++i)
            for (int t = 0; t < 2; ++t) {
              const SubDev &d = P.subs[i];
              const long long M = d.M, r0 = (long long)jb * INVB;
              if (d.M <= INVB || r0 >= M) continue;
              CholDesc b = P.cdesc[c0 + 2 * (i - w0) + t];
              b.g += r0 * M + r0;
              b.v += r0 * M + r0;
              b.M = int(std::min<long long>(INVB, M - r0));
              b.ld = d.M;
              b.mode = 0;
              b.ridge = 0;
              b.shift_kind = 0;
              b.inv_block = 0;
              b.epsout = -1;
              b.z = -1;
              P.cdesc.push_back(b);
            }
          chol_step(cb0);
          for (int part = 0; part < 2; ++part) {
            GemmPhase ph = phase_begin();
            for (int i = w0; i < w1; ++i)
              for (int t = 0; t < 2; ++t) {
                const SubDev &d = P.subs[i];
                const long long M = d.M, r0 = (long long)jb * INVB, r1 = r0 + INVB, rest = M - r1;
                if (d.M <= INVB || rest <= 0) continue;
                const CholDesc &c = P.cdesc[c0 + 2 * (i - w0) + t];
                const int bj = INVB;
                if (part == 0)  // panel: V_rr^T A[r, r+1:]
                  add(ph, c.v + r0 * M + r0, c.g + r0 * M + r1, c.g + r0 * M + r1, bj, int(rest), bj, d.M, d.M,
                      d.M, 1, 0, 0, 1.0, 0.0);
                else            // trailing update of the upper triangle
                  add(ph, c.g + r0 * M + r1, c.g + r0 * M + r1, c.g + r1 * M + r1, int(rest), int(rest), bj, d.M,
                      d.M, d.M, 1, 0, 0, -1.0, 1.0, true);
              }
            gemm_step(ph, lv_factor, 4);
          }
        }
      } else {
        chol_step(c0);
      }
      if (blocked_inv && P.cdesc[c0].prec != 1) {
        // block back substitution, block rows from the bottom:
        //   T = R[r, r+1:] V[r+1:, r+1:] ;  V[r, r+1:] = -V_rr T
        int maxnb = 0;
        for (int i = w0; i < w1; ++i) maxnb = std::max(maxnb, (P.subs[i].M + INVB - 1) / INVB);
        for (int st = 0; st + 2 <= maxnb; ++st) {
          // (a phase's descriptors and tiles are contiguous: build one phase at a time)
          for (int half = 0; half < 2; ++half) {
            GemmPhase ph = phase_begin();
            for (int i = w0; i < w1; ++i)
              for (int t = 0; t < 2; ++t) {
                const SubDev &d = P.subs[i];
                const int nbi = (d.M + INVB - 1) / INVB;
                const int r = nbi - 2 - st;
                if (d.M <= INVB || r < 0) continue;
                const long long M = d.M, r0 = (long long)r * INVB, r1 = r0 + INVB, n1 = M - r1;
                const long long V = (last && !P.polish) ? scr[i].v[t].V3 : vk(i, t, k);
                const long long Tb = scr[i].v[t].W32;  // INVB x n1 scratch (FP64 passes leave it free)
                if (half == 0)
                  add(ph, scr[i].v[t].G + r0 * M + r1, V + r1 * M + r1, Tb, INVB, int(n1), int(n1), d.M, d.M,
                      int(n1), 0, 0, GEMM_B_UPPER, 1.0, 0.0);
                else
                  add(ph, V + r0 * M + r0, Tb, V + r0 * M + r1, INVB, int(n1), INVB, d.M, int(n1), d.M, 0, 0,
                      GEMM_A_UPPER, -1.0, 0.0);
              }
            gemm_step(ph, lv_factor, 4);
          }
        }
        if (k == 0) {
          const int m0 = int(P.mdesc.size());
          for (int i = w0; i < w1; ++i)
            for (int t = 0; t < 2; ++t)
              if (P.subs[i].M > INVB)
                P.mdesc.push_back(MatopDesc{vk(i, t, 0), P.o_eps + 2 * i + t, zk(i, t, 0), P.subs[i].M, 5, 2 * i + t, -1});
          if ((int)P.mdesc.size() > m0) matop_step(m0);  // Z1 = eps V1
        }
      }
      if (last) break;
      // Q_{k+1} = Q_k V_k, Z_{k+1} = Z_k V_k, T_k = T_{k-1} V_k (T_0 = V_0)
      {
        GemmPhase ph = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph, qk(i, t, k), vk(i, t, k), qk(i, t, k + 1), d.m, d.M, d.M, d.M, d.M, d.M, 0, 0, GEMM_B_UPPER,
                1.0, 0.0);
            if (k > 0)
              add(ph, zk(i, t, k - 1), vk(i, t, k), zk(i, t, k), d.M, d.M, d.M, d.M, d.M, d.M, 0, 0,
                  GEMM_A_UPPER | GEMM_B_UPPER, 1.0, 0.0);
          }
        gemm_step(ph, lv_update, 2);
      }
      if (k > 0) {
        GemmPhase ph = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph, tk(i, t, k - 1), vk(i, t, k), tk(i, t, k), d.M, d.M, d.M, d.M, d.M, d.M, 0, 0,
                GEMM_A_UPPER | GEMM_B_UPPER, 1.0, 0.0);
          }
        gemm_step(ph, lv_factor, 4);
      }
      // the Gram of pass k+1: G = Q^T Q, then G += Z^T Z (Z upper triangular)
      const int lv = (fp32 && k + 1 < N) ? lv_shifted32 : lv_exact;
      {
        GemmPhase ph = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph, qk(i, t, k + 1), qk(i, t, k + 1), scr[i].v[t].G, d.M, d.M, d.m, d.M, d.M, d.M, 1, 0, 0, 1.0,
                0.0, true);
          }
        gemm_step(ph, lv, 1);
        GemmPhase ph2 = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph2, zk(i, t, k), zk(i, t, k), scr[i].v[t].G, d.M, d.M, d.M, d.M, d.M, d.M, 1, 0, GEMM_B_UPPER,
                1.0, 1.0, true);
          }
        gemm_step(ph2, lv, 1);
      }
    }
    if (P.polish) {
      // The last pass leaves a Gram close to I.  FP32 scheme: with V_l the FP32
      // Cholesky inverse of G, E = V_l^T G V_l - I; series scheme (no last
      // Cholesky): E = G - I.  Then W = I - E/2 + 3/8 E^2 - 5/16 E^3, the series
      // of (I + E)^{-1/2}, and V3 = V_l W (or W): [Q; Z] V3 is orthonormal to
      // O(|E|^4).
      auto H = [&](int i, int t) { return zk(i, t, N - 1); };  // free after the last Gram
      auto E = [&](int i, int t) { return zk(i, t, N); };
      auto E2 = [&](int i, int t) { return vk(i, t, N - 1); };
      auto E3 = [&](int i, int t) { return tk(i, t, N); };      // the accumulated product is tk(N-1)
      int m0 = int(P.mdesc.size());
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t)
          P.mdesc.push_back(MatopDesc{scr[i].v[t].G, 0, scr[i].v[t].G, P.subs[i].M, 2, 2 * i + t, -1});
      if (!series)
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) P.mdesc.push_back(MatopDesc{0, 0, E(i, t), P.subs[i].M, 0, 2 * i + t, -1});
      matop_step(m0);  // G lower = G upper ; E = -I
      if (series) {
        m0 = int(P.mdesc.size());
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t)
            P.mdesc.push_back(MatopDesc{scr[i].v[t].G, 0, E(i, t), P.subs[i].M, 4, 2 * i + t, -1});
        matop_step(m0);  // E = G - I
      } else {
        GemmPhase ph = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph, scr[i].v[t].G, vk(i, t, N), H(i, t), d.M, d.M, d.M, d.M, d.M, d.M, 0, 0, GEMM_B_UPPER, 1.0, 0.0);
          }
        gemm_step(ph, lv_exact, 4);
        GemmPhase ph2 = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph2, vk(i, t, N), H(i, t), E(i, t), d.M, d.M, d.M, d.M, d.M, d.M, 1, 0, 0, 1.0, 1.0);
          }
        gemm_step(ph2, lv_exact, 1);
      }
      GemmPhase ph3 = phase_begin();
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t) {
          const SubDev &d = P.subs[i];
          add(ph3, E(i, t), E(i, t), E2(i, t), d.M, d.M, d.M, d.M, d.M, d.M, 0, 0, 0, 1.0, 0.0);
        }
      gemm_step(ph3, lv_small, 0);
      GemmPhase ph5 = phase_begin();
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t) {
          const SubDev &d = P.subs[i];
          add(ph5, E2(i, t), E(i, t), E3(i, t), d.M, d.M, d.M, d.M, d.M, d.M, 0, 0, 0, 1.0, 0.0);
        }
      gemm_step(ph5, lv_tiny, 0);
      m0 = int(P.mdesc.size());
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t)
          P.mdesc.push_back(MatopDesc{E(i, t), E2(i, t), series ? scr[i].v[t].V3 : E2(i, t), P.subs[i].M, 1,
                                      2 * i + t, E3(i, t)});
      matop_step(m0);  // W = I - E/2 + 3/8 E^2 - 5/16 E^3 (checks |E|)
      if (!series) {
        GemmPhase ph4 = phase_begin();
        for (int i = w0; i < w1; ++i)
          for (int t = 0; t < 2; ++t) {
            const SubDev &d = P.subs[i];
            add(ph4, vk(i, t, N), E2(i, t), scr[i].v[t].V3, d.M, d.M, d.M, d.M, d.M, d.M, 0, 0, GEMM_A_UPPER, 1.0,
                0.0);
          }
        gemm_step(ph4, lv_exact, 4);
      }
    }
    // R^{-1} = T_{N-1} V3
    {
      GemmPhase ph = phase_begin();
      for (int i = w0; i < w1; ++i)
        for (int t = 0; t < 2; ++t) {
          const SubDev &d = P.subs[i];
          add(ph, tk(i, t, N - 1), scr[i].v[t].V3, scr[i].v[t].V, d.M, d.M, d.M, d.M, d.M, d.M, 0, 0,
              GEMM_A_UPPER | TU, 1.0, 0.0);
        }
      gemm_step(ph, lv_factor, 4);
    }
    // Q_Gamma = Q_N[Gamma rows] V3 ; Q-bar_Delta = Q-bar_N[Delta rows] V3-bar ; A_m V ; A-bar V-bar
    {
      GemmPhase ph = phase_begin();
      for (int i = w0; i < w1; ++i) {
        const SubDev &d = P.subs[i];
        const long long M = d.M;
        add(ph, qk(i, 0, N) + (long long)(d.nI + d.nB) * M, scr[i].v[0].V3, d.oQG, d.nG, d.M, d.M, d.M, d.M, d.M,
            0, 0, TU, 1.0, 0.0);
        add(ph, qk(i, 1, N) + (long long)(d.m - d.nDl) * M, scr[i].v[1].V3, scr[i].QbD, d.nDl, d.M, d.M, d.M,
            d.M, d.M, 0, 0, TU, 1.0, 0.0);
        add(ph, d.oA, d.oV, scr[i].AV, d.nG, d.M, d.M, d.M, d.M, d.M, 0, 0, TU, 1.0, 0.0);
        add(ph, d.oAbar, scr[i].v[1].V, scr[i].AbV, d.nDl, d.M, d.M, d.M, d.M, d.M, 0, 0, TU, 1.0, 0.0);
      }
      gemm_step(ph, lv_ops, 8);
    }
    // Lambda, Lambda^T, Psi, K^+ E_Gamma, Phi, Phi^T
    {
      GemmPhase ph = phase_begin();
      for (int i = w0; i < w1; ++i) {
        const SubDev &d = P.subs[i];
        add(ph, scr[i].AV, d.oQG, d.oLam, d.nG, d.nG, d.M, d.M, d.M, d.nG, 0, 1, 0, 1.0, 0.0);
        add(ph, d.oQG, scr[i].AV, d.oLamT, d.nG, d.nG, d.M, d.M, d.M, d.nG, 0, 1, 0, 1.0, 0.0);
        add(ph, d.oQG, d.oQG, d.oPsi, d.nG, d.nG, d.M, d.M, d.M, d.nG, 0, 1, 0, 1.0, 0.0);
        add(ph, d.oV, d.oQG, d.oKpE, d.M, d.nG, d.M, d.M, d.M, d.nG, 0, 1, TA, 1.0, 0.0);
        add(ph, scr[i].AbV, scr[i].QbD, d.oPhi, d.nDl, d.nDl, d.M, d.M, d.M, d.nDl, 0, 1, 0, 1.0, 0.0);
        add(ph, scr[i].QbD, scr[i].AbV, d.oPhiT, d.nDl, d.nDl, d.M, d.M, d.M, d.nDl, 0, 1, 0, 1.0, 0.0);
      }
      gemm_step(ph, lv_ops, 8);
    }
  }
  P.ph_coarse = int(P.setup_gemm.size());
  fp64_tiles = true;
  // coarse: 11: S_Pi += D^T D ; 12: Sinv = V_Pi V_Pi^T ; 13: C1 = Sinv D^T, C3 = D Sinv ;
  //         14: C2 = I - D C1.  A small coarse space takes 16 x 16 tiles, so that
  //         these products spread over more than a few SMs.
  if (n_pi > 0) {
    const int ct = n_pi <= 192 ? 16 : 64;
    GemmPhase a = phase_begin(0, ct);
    add(a, P.o_Dpp, P.o_Dpp, P.o_Spi, n_pi, n_pi, n_pi, n_pi, n_pi, n_pi, 1, 0, 0, 1.0, 1.0);
    push(a);
    GemmPhase b = phase_begin(0, ct);
    add(b, P.o_Vpi, P.o_Vpi, P.o_Sinv, n_pi, n_pi, n_pi, n_pi, n_pi, n_pi, 0, 1, GEMM_A_UPPER, 1.0, 0.0);
    push(b);
    GemmPhase c = phase_begin(0, ct);
    add(c, P.o_Sinv, P.o_Dpp, P.o_C1, n_pi, n_pi, n_pi, n_pi, n_pi, n_pi, 0, 1, 0, 1.0, 0.0);
    add(c, P.o_Dpp, P.o_Sinv, P.o_C3, n_pi, n_pi, n_pi, n_pi, n_pi, n_pi, 0, 0, 0, 1.0, 0.0);
    push(c);
    GemmPhase e = phase_begin(0, ct);
    add(e, P.o_Dpp, P.o_C1, P.o_C2, n_pi, n_pi, n_pi, n_pi, n_pi, n_pi, 0, 0, 0, -1.0, 1.0);
    push(e);
  } else {
    for (int k = 0; k < 4; ++k) P.setup_gemm.push_back(GemmPhase{0, 0, 0, 0, 0, 64});
  }
  P.ph_solve = int(P.setup_gemm.size());
  // solve phases: 15: T = Q2[IB rows]^T F ; 16: Qtf = V3^T T ; 17: y = V Qtf, p = Q_Gamma Qtf ;
  //               18: a = A_m y ; 19: u_eval = Eval c
  {
    GemmPhase a = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(a, d.oX, d.oF, d.oT, d.M, R, d.nI + d.nB, d.M, R, R, 1, 0, 0, 1.0, 0.0);
    }
    push(a);
    GemmPhase b = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(b, d.oV3, d.oT, d.oQtf, d.M, R, d.M, d.M, R, R, 1, 0, 0, 1.0, 0.0);
    }
    push(b);
    GemmPhase c = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(c, d.oV, d.oQtf, d.oY, d.M, R, d.M, d.M, R, R, 0, 0, TA, 1.0, 0.0);
      add(c, d.oQG, d.oQtf, d.oP, d.nG, R, d.M, d.M, R, R, 0, 0, 0, 1.0, 0.0);
    }
    push(c);
    GemmPhase e = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(e, d.oA, d.oY, d.oAy, d.nG, R, d.M, d.M, R, R, 0, 0, 0, 1.0, 0.0);
    }
    push(e);
    GemmPhase f = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(f, d.oEval, d.oC, d.oU, d.nE, R, d.M, d.M, R, R, 0, 0, 0, 1.0, 0.0);
    }
    push(f);
  }

  for (size_t q = 0; q < P.setup_gemm.size(); ++q) {
    double f = 0.0;
    for (int k = 0; k < P.setup_gemm[q].ndesc; ++k) f += P.gemm_flops[P.setup_gemm[q].desc0 + k];
    P.phase_flops.push_back(f);
  }
  P.ph_adj = int(P.setup_gemm.size());
  // adjoint phases: 20: c-bar += Eval^T u-bar ; 21: y-bar += A_m^T a-bar ; 22: Qtf-bar = Q_Gamma^T p-bar ;
  //                 23: Qtf-bar += V^T y-bar ; 24: T-bar = V3 Qtf-bar ; 25: F-bar = Q2[IB rows] T-bar
  {
    GemmPhase a = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(a, d.oEval, d.oU, d.oC, d.M, R, d.nE, d.M, R, R, 1, 0, 0, 1.0, 1.0);
    }
    push(a);
    GemmPhase b = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(b, d.oA, d.oAy, d.oY, d.M, R, d.nG, d.M, R, R, 1, 0, 0, 1.0, 1.0);
    }
    push(b);
    GemmPhase c = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(c, d.oQG, d.oP, d.oQtf, d.M, R, d.nG, d.M, R, R, 1, 0, 0, 1.0, 0.0);
    }
    push(c);
    GemmPhase e = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(e, d.oV, d.oY, d.oQtf, d.M, R, d.M, d.M, R, R, 1, 0, 0, 1.0, 1.0);
    }
    push(e);
    GemmPhase f = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(f, d.oV3, d.oQtf, d.oT, d.M, R, d.M, d.M, R, R, 0, 0, 0, 1.0, 0.0);
    }
    push(f);
    GemmPhase g2 = phase_begin(1);
    for (int i = 0; i < n_sub; ++i) {
      const SubDev &d = P.subs[i];
      add(g2, d.oX, d.oT, d.oF, d.nI + d.nB, R, d.M, d.M, R, R, 0, 0, 0, 1.0, 0.0);
    }
    push(g2);
  }

  // ---- coarse Cholesky
  P.chol_coarse.desc0 = int(P.cdesc.size());
  if (n_pi > 0) {
    CholDesc c;
    std::memset(&c, 0, sizeof(c));
    c.g = P.o_SpiR;  // a copy of S_Pi, factored in place
    c.v = P.o_Vpi;
    c.z = -1;
    c.w = -1;
    c.epsout = -1;
    c.M = n_pi;
    c.m = n_pi;
    c.status = 2 * n_sub;
    P.cdesc.push_back(c);
  }
  P.chol_coarse.ndesc = int(P.cdesc.size()) - P.chol_coarse.desc0;
  for (const auto &c : P.cdesc) {
    if (c.mode == 1) continue;  // diagonal additions only
    double f = 2.0 * c.M * (double)c.M * c.M / 3.0;  // factor + inverse
    if (c.inv_block > 0) {  // factor + the diagonal blocks of the inverse
      f = c.M * (double)c.M * c.M / 3.0;
      for (int b0 = 0; b0 < c.M; b0 += c.inv_block) {
        const double bs = std::min(c.inv_block, c.M - b0);
        f += bs * bs * bs / 3.0;
      }
    }
    P.chol_flops += f;
    if (c.prec == 1) P.chol_flops32 += f;
  }

  // ---- tensor-core emulation tables (precision MIXED)
  if (o.precision == DDELM_PREC_MIXED) {
    P.mixed = true;
    P.tc_tiles = o.tc_tiles;
    P.autotune = o.autotune != 0;
    if (build_mixed(P, cur) != DDELM_OK) {
      const std::string e = P.err.empty() ? std::string("mixed plan") : P.err;
      return fail(e.c_str());
    }
  }
  // ---- scale gradient: tables and buffers (inside the free setup scratch)
  if (build_scale(P, cur) != DDELM_OK) {
    const std::string e = P.err.empty() ? std::string("scale plan") : P.err;
    return fail(e.c_str());
  }
  P.n_dbl = cur;

  // ---- bounds of every access the kernels make (an error here, not a fault there)
  {
    const long long N = P.n_dbl;
    auto in = [&](long long off, long long len) { return off >= 0 && len >= 0 && off + len <= N; };
    for (const auto &d : P.gdesc) {
      const long long alen = d.ta ? (long long)(d.k - 1) * d.lda + d.m : (long long)(d.m - 1) * d.lda + d.k;
      const long long blen = d.tb ? (long long)(d.n - 1) * d.ldb + d.k : (long long)(d.k - 1) * d.ldb + d.n;
      const long long clen = (long long)(d.m - 1) * d.ldc + d.n;
      if (d.k > 0 && (!in(d.a, alen) || !in(d.b, blen))) return fail("internal: GEMM operand out of bounds");
      if (!in(d.c, clen)) return fail("internal: GEMM output out of bounds");
      if ((d.ta ? d.lda < d.m : d.lda < d.k) || (d.tb ? d.ldb < d.k : d.ldb < d.n) || d.ldc < d.n)
        return fail("internal: GEMM leading dimension");
    }
    for (const auto &t : P.gtile)
      if (t.desc < 0 || t.desc >= (int)P.gdesc.size()) return fail("internal: GEMM tile");
    auto phase_ok = [&](const GemmPhase &ph) {  // a phase's tiles use only its own descriptors
      for (int q = ph.tile0; q < ph.tile0 + ph.ntile; ++q)
        if (q < 0 || q >= (int)P.gtile.size() || P.gtile[q].desc < ph.desc0 || P.gtile[q].desc >= ph.desc0 + ph.ndesc)
          return false;
      return true;
    };
    for (const auto &ph : P.setup_gemm)
      if (!phase_ok(ph)) return fail("internal: GEMM phase tiles");
    for (const auto &ph : P.sc_coarse)
      if (!phase_ok(ph)) return fail("internal: GEMM phase tiles");
    for (const auto &w : P.sc_wave)
      for (const auto &ph : w)
        if (!phase_ok(ph)) return fail("internal: GEMM phase tiles");
    for (const auto &dd : P.dots) {
      const long long al = dd.rows > 0 ? (long long)(dd.rows - 1) * dd.lda + dd.cols : 0;
      const long long bl = dd.rows > 0 ? (long long)(dd.rows - 1) * dd.ldb + dd.cols : 0;
      if (!in(dd.a, al) || !in(dd.b, bl) || dd.sub < 0 || dd.sub >= n_sub || dd.lda < dd.cols || dd.ldb < dd.cols)
        return fail("internal: dot product bounds");
    }
    for (const auto &c : P.cdesc) {
      // a diagonal block with leading dimension ld spans (M - 1) ld + M entries
      const long long mm = c.ld > 0 ? (long long)(c.M - 1) * c.ld + c.M : (long long)c.M * c.M;
      if (c.ld > 0 && (c.ld < c.M || c.mode != 0 || c.ridge || c.shift_kind || c.prec != 0))
        return fail("internal: Cholesky block");
      if (!in(c.g, mm) || !in(c.v, mm) || (c.z >= 0 && !in(c.z, mm)) || (c.prec == 1 && !in(c.w, mm)))
        return fail("internal: Cholesky bounds");
      if (c.prec == 1 && c.band != 0) return fail("internal: banded FP32 Cholesky");
      if (c.epsout >= 0 && !in(c.epsout, 1)) return fail("internal: eps slot");
      if (c.status < 0 || c.status > 2 * n_sub) return fail("internal: status slot");
    }
    for (const auto &cv : P.conv)
      if (!in(cv.src, cv.n) || cv.dst < 0 || cv.dst + cv.n > P.n_f32) return fail("internal: FP32 copy bounds");
    for (const auto &md : P.mdesc) {
      const long long mm = (long long)md.M * md.M;
      if (!in(md.c, mm) || (md.op == 1 && (!in(md.a, mm) || !in(md.b, mm) || (md.d >= 0 && !in(md.d, mm)))) ||
          ((md.op == 3 || md.op == 4 || md.op == 5) && !in(md.a, mm)) || (md.op == 5 && !in(md.b, 1)) ||
          md.op < 0 || md.op > 5 ||
          md.status < 0 || md.status >= 2 * n_sub)
        return fail("internal: matrix operation bounds");
    }
    if ((int)P.wave_row0.size() != P.n_waves + 1 || P.wave_row0[P.n_waves] > (int)P.rows.size())
      return fail("internal: wave rows");
    for (const auto &r : P.rows) {
      const long long M = P.subs[r.sub].M;
      if (!in(r.out0, M) || (r.out1 >= 0 && !in(r.out1, M))) return fail("internal: row output bounds");
      if (r.kind == ROW_DELTA && (!in(r.out2, M) || !in(r.out3, M) || (r.ca >= 0 && !in(r.ca, M)) ||
                                  (r.cb >= 0 && !in(r.cb, M))))
        return fail("internal: Delta row bounds");
      if (r.kind == ROW_AM) {
        if (!in(r.ca, M)) return fail("internal: corner row bounds");
        for (int t = 0; t < 2; ++t)
          if (r.am_e[t] < 0 || (r.am_e[t] > 0 && !in(r.am_f[t], (long long)r.am_e[t] * M)))
            return fail("internal: A_m flux row bounds");
      }
    }
    for (const auto &d : P.subs) {
      const long long M = d.M, m = d.m;
      if (!in(d.oX, m * M) || !in(d.oK, m * M) || !in(d.oKb, m * M) || !in(d.oY1, m * M) || !in(d.oY1b, m * M) ||
          !in(d.oA, d.nG * M) || !in(d.oAbar, d.nDl * M) || !in(d.oEval, d.nE * M) ||
          !in(d.oLam, (long long)d.nG * d.nG) || !in(d.oLamT, (long long)d.nG * d.nG) ||
          !in(d.oPsi, (long long)d.nG * d.nG) || !in(d.oPhi, (long long)d.nDl * d.nDl) ||
          !in(d.oPhiT, (long long)d.nDl * d.nDl) || !in(d.oKpE, M * d.nG) || !in(d.oY, M * R) ||
          !in(d.oAy, d.nG * (long long)R) || !in(d.oP, d.nG * (long long)R) || !in(d.oC, M * R) ||
          !in(d.oU, (long long)d.nE * R) || !in(d.oF, (long long)(d.nI + d.nB) * R))
        return fail("internal: subdomain buffer bounds");
      if (d.w_off + d.M > sumM || d.int_off + d.nI > sumI || d.eval_off + d.nE > sumE)
        return fail("internal: packed input bounds");
      if (d.loc_off + d.nG > sum_nG) return fail("internal: local slab bounds");
      for (int k = 0; k < d.nPi; ++k)
        if (I[d.gpi_off + k] < 0 || I[d.gpi_off + k] >= n_pi) return fail("internal: R_Pi map");
      for (int k = 0; k < d.nDl; ++k)
        if (I[d.gdl_off + k] < 0 || I[d.gdl_off + k] >= nd) return fail("internal: R_Delta map");
      for (int k = 0; k < d.nB; ++k)
        if (I[d.bnd_off + k] < 0 || I[d.bnd_off + k] >= nb) return fail("internal: boundary map");
    }
    for (int p = 0; p < n_pi; ++p)
      for (int o = 0; o < 4; ++o) {
        const int s = I[P.o_pi_own + 8 * p + 2 * o], a = I[P.o_pi_own + 8 * p + 2 * o + 1];
        if (s >= 0 && (s >= n_sub || a < 0 || a >= P.subs[s].nPi)) return fail("internal: Pi owner map");
      }
    for (int p = 0; p < nd; ++p)
      for (int o = 0; o < 4; ++o) {
        const int s = I[P.o_dl_own + 8 * p + 2 * o], a = I[P.o_dl_own + 8 * p + 2 * o + 1];
        if (o < 2 && s < 0) return fail("internal: Delta point without two owners");
        if (s >= 0 && (s >= n_sub || a < 0 || a >= P.subs[s].nDl)) return fail("internal: Delta owner map");
        const int r = I[P.o_dl_rows + 4 * p + o];
        if ((s < 0) != (r < 0) || r >= P.sum_nG) return fail("internal: Delta slab rows");
      }
    if (P.o_dl_rows % 4 || P.o_gam_rows % 4) return fail("internal: int4 table alignment");
    for (int b = 0; b < nb; ++b) {
      const int s0 = I[P.o_bnd_own + 4 * b];
      if (s0 < 0) return fail("internal: boundary point without owner");
      for (int o = 0; o < 2; ++o) {
        const int s = I[P.o_bnd_own + 4 * b + 2 * o], a = I[P.o_bnd_own + 4 * b + 2 * o + 1];
        if (s >= 0 && (s >= n_sub || a < 0 || a >= P.subs[s].nB)) return fail("internal: boundary owner map");
      }
    }
    for (const auto &s : P.sdesc) {
      const long long len = s.trans ? (long long)(s.K - 1) * s.ld + s.R : (long long)(s.R - 1) * s.ld + s.K;
      if (!in(s.x, len) || !in(s.scale, s.R)) return fail("internal: slice source bounds");
      if ((s.out + (long long)s.S * s.Rpad * s.Kpad) * 2 > (long long)P.bytes_slices)
        return fail("internal: slice buffer bounds");
      if (s.Rpad % 128 || s.Kpad % 64 || s.Rpad < s.R || s.Kpad < s.K) return fail("internal: slice padding");
    }
    for (const auto &od : P.odesc) {
      if (!in(od.c, (long long)(od.m - 1) * od.ldc + od.n)) return fail("internal: tensor-core GEMM output bounds");
      if (od.tmapA < 0 || od.tmapA >= (int)P.sdesc.size() || od.tmapB < 0 || od.tmapB >= (int)P.sdesc.size())
        return fail("internal: tensor map index");
      if (od.RpadA != P.sdesc[od.tmapA].Rpad || od.RpadB != P.sdesc[od.tmapB].Rpad ||
          od.Kpad != P.sdesc[od.tmapA].Kpad || od.Kpad != P.sdesc[od.tmapB].Kpad || od.S > P.sdesc[od.tmapA].S ||
          od.S > P.sdesc[od.tmapB].S || od.kc % 64 || od.kc > 1024)
        return fail("internal: tensor-core GEMM shape");
    }
    for (const auto &ph : P.oz_phase) {
      auto width_ok = [](int bn) { return bn == 48 || bn == 64 || bn == 128; };
      if (!width_ok(ph.bn)) return fail("internal: tensor-core tile width");
      if (ph.ntile_alt > 0 && (!width_ok(ph.bn_alt) || ph.bn_alt == ph.bn))
        return fail("internal: tensor-core alternative width");
      if (ph.ntile > 0 && (ph.bn == 48 || (ph.ntile_alt > 0 && ph.bn_alt == 48)) &&
          (P.sdesc[ph.slice0].S < 1 || P.sdesc[ph.slice0].S > 10))
        return fail("internal: all-levels tile levels");
      // both tile lists (the rule's and the autotuner's alternative)
      for (int which = 0; which < 2; ++which) {
        const int t0 = which ? ph.tile0_alt : ph.tile0, nt = which ? ph.ntile_alt : ph.ntile;
        const int bn = which ? ph.bn_alt : ph.bn;
        if (t0 < 0 || (size_t)t0 + nt > P.otile.size()) return fail("internal: tensor-core tile list");
        for (int q = t0; q < t0 + nt; ++q) {
          const OzTile &t = P.otile[q];
          if (t.desc < ph.desc0 || t.desc >= ph.desc0 + ph.ndesc) return fail("internal: tensor-core tile");
          const OzDesc &od = P.odesc[t.desc];
          // 48-wide tiles may reach past the padded rows of B: the copy's
          // bounds are the tensor map's R rows, past which it fills zeros
          if ((t.tm + 1) * 128 > od.RpadA || (bn == 48 ? t.tn * bn >= od.n : (t.tn + 1) * bn > od.RpadB))
            return fail("internal: tensor-core tile box");
          const int bk = bn == 48 ? 32 : 64;
          if (t.kb0 < 0 || t.kb1 < t.kb0 || t.kb1 * bk > od.Kpad) return fail("internal: tensor-core tile k range");
        }
      }
    }
    const long long cg_need = 12LL * std::max(nd, 1) * R + 14LL * std::max(n_pi, 1) * R + 2048 * 32;
    if (!in(P.o_cg, cg_need) || !in(P.o_loc, 9LL * sum_nG * R) || !in(P.o_status, 4LL * n_sub + 64))
      return fail("internal: CG region bounds");
    const long long np2 = (long long)std::max(n_pi, 1) * std::max(n_pi, 1);
    for (long long o : {P.o_Dpp, P.o_Spi, P.o_Vpi, P.o_Sinv, P.o_C1, P.o_C2, P.o_C3, P.o_SpiR})
      if (!in(o, np2)) return fail("internal: coarse bounds");
  }

  // ---- table region (bytes), then the double region
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  P.off_subs = off;
  off = al(off + P.subs.size() * sizeof(SubDev));
  P.off_rows = off;
  off = al(off + std::max<size_t>(P.rows.size(), 1) * sizeof(SpecialRow));
  P.off_gdesc = off;
  off = al(off + std::max<size_t>(P.gdesc.size(), 1) * sizeof(GemmDesc));
  P.off_gtile = off;
  off = al(off + std::max<size_t>(P.gtile.size(), 1) * sizeof(GemmTile));
  P.off_cdesc = off;
  off = al(off + std::max<size_t>(P.cdesc.size(), 1) * sizeof(CholDesc));
  P.off_conv = off;
  off = al(off + std::max<size_t>(P.conv.size(), 1) * sizeof(ConvSeg));
  P.off_mdesc = off;
  off = al(off + std::max<size_t>(P.mdesc.size(), 1) * sizeof(MatopDesc));
  P.off_ints = off;
  off = al(off + std::max<size_t>(P.ints.size(), 1) * sizeof(int));
  P.off_sdesc = off;
  off = al(off + std::max<size_t>(P.sdesc.size(), 1) * sizeof(SliceDesc));
  P.off_odesc = off;
  off = al(off + std::max<size_t>(P.odesc.size(), 1) * sizeof(OzDesc));
  P.off_otile = off;
  off = al(off + std::max<size_t>(P.otile.size(), 1) * sizeof(OzTile));
  P.off_tmaps = off;
  off = al(off + std::max<size_t>(P.sdesc.size(), 1) * 3 * 128);  // three tensor maps per slice buffer
  P.off_ssubs = off;
  off = al(off + std::max<size_t>(P.ssubs.size(), 1) * sizeof(SubDev));
  P.off_srows = off;
  off = al(off + std::max<size_t>(P.srows.size(), 1) * sizeof(SpecialRow));
  P.off_scsub = off;
  off = al(off + std::max<size_t>(P.scsub.size(), 1) * sizeof(ScaleSub));
  P.off_dots = off;
  off = al(off + std::max<size_t>(P.dots.size(), 1) * sizeof(DotDesc));
  P.bytes_tables = off;
  P.off_dbl = off;
  off = al(off + (size_t)P.n_dbl * sizeof(double));
  P.off_slices = off;
  P.bytes_total = off + P.bytes_slices;
  P.sz.workspace_bytes = P.bytes_total;
  P.sz.upload_bytes = P.bytes_tables + sizeof(double) * (size_t)(3 * sumM + 2 * sumI) +
                      (pr.op == DDELM_OP_DIFFUSION ? sizeof(double) * (size_t)(3 * sumI) : 0);
  return DDELM_OK;
}

}  // namespace ddelm
