// Scale gradient dL/ds, the per-subdomain stages (the layout and the GEMM phases
// are in scale_plan.cpp; the interface vectors come from mode 4 of the
// persistent kernel in cg.cu):
//   gather  -- the factored cotangents of the local operators from the bank of
//              interface vectors (restricted to the subdomain), and the initial
//              values of the accumulated products;
//   dots    -- the block dot products sum(L o (dX R)) of the contraction;
//   total   -- per subdomain the contraction plus the two ridge terms
//              d(eps^2)/ds = 2 eps_rel^2 <K, dK> / M times the eps^2 cotangent,
//              then the sum over subdomains in a fixed order.
#include <algorithm>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

struct GatherArgs {
  const SubDev *subs;
  const ScaleSub *sc;
  const int *ints;
  double *db;
  int sub0, R, n_pi, n_dl;
  int JL, JP, JF, Jc, NK, NAG;
  long long bkd, bkp, Db, SPb;
  double theta;
};

// Local restriction of bank vectors: rows a < nPi from Pi slot sp (scaled by
// fp), rows a >= nPi from Delta slot sd (scaled by fd); slot < 0: zero.
__device__ __forceinline__ double lrow(const GatherArgs &g, const SubDev &d, int a, int k, int sp, double fp, int sd,
                                       double fd) {
  const long long nd = g.n_dl > 0 ? g.n_dl : 1, np = g.n_pi > 0 ? g.n_pi : 1;
  if (a < d.nPi) {
    if (sp < 0) return 0.0;
    const int gp = g.ints[d.gpi_off + a];
    return fp * g.db[g.bkp + (long long)sp * np * g.R + (long long)gp * g.R + k];
  }
  if (sd < 0) return 0.0;
  const int gd = g.ints[d.gdl_off + a - d.nPi];
  return fd * g.db[g.bkd + (long long)sd * nd * g.R + (long long)gd * g.R + k];
}

__global__ void __launch_bounds__(256) scale_gather_kernel(GatherArgs g) {
  const int i = g.sub0 + blockIdx.x;
  const SubDev d = g.subs[i];
  const ScaleSub q = g.sc[i];
  const int R = g.R, M = d.M, m = d.m, nG = d.nG, nPi = d.nPi, nDl = d.nDl;
  const int JL = g.JL, JP = g.JP, JF = g.JF, Jc = g.Jc, NK = g.NK, NAG = g.NAG;
  double *db = g.db;
  const int np = g.n_pi;
  // coarse pair columns: Lambda-bar_PiPi += D-bar block, Psi-bar_PiPi -= S-bar block
  auto coarse = [&](long long mat, double sgn, int cc, int b) -> double {
    if (cc >= nPi || b >= nPi) return 0.0;
    const int gc = g.ints[d.gpi_off + cc], gb = g.ints[d.gpi_off + b];
    return sgn * db[mat + (long long)gc * np + gb];
  };
  // Bc = [ell | WL | WP]
  for (int e = threadIdx.x; e < nG * Jc; e += blockDim.x) {
    const int a = e / Jc, col = e % Jc;
    double v;
    if (col < R) {
      v = lrow(g, d, a, col, SP_MPIF, 1.0, SD_MU, 1.0);
    } else if (col < R + 4 * R) {
      const int grp = (col - R) / R, k = (col - R) % R;
      if (grp == 0) v = lrow(g, d, a, k, -1, 0.0, SD_BB, 1.0);
      else if (grp == 1) v = lrow(g, d, a, k, -1, 0.0, SD_MU, 1.0);
      else if (grp == 2) v = lrow(g, d, a, k, SP_RNUB, 1.0, SD_BB, 1.0);
      else v = lrow(g, d, a, k, SP_PIC, 1.0, SD_MU, -1.0);
    } else if (col < R + JL) {
      v = coarse(g.Db, 1.0, col - 5 * R, a);
    } else if (col < R + JL + 2 * R) {
      const int grp = (col - R - JL) / R, k = (col - R - JL) % R;
      v = grp == 0 ? lrow(g, d, a, k, SP_PID, 1.0, SD_MU, 1.0) : lrow(g, d, a, k, -1, 0.0, SD_MU, 1.0);
    } else {
      v = coarse(g.SPb, -1.0, col - R - JL - 2 * R, a);
    }
    db[q.Bc + (long long)a * Jc + col] = v;
  }
  // LA = [PL | 0 | a-bar] and LG = [0 | PP | p-bar]
  for (int e = threadIdx.x; e < nG * NAG; e += blockDim.x) {
    const int a = e / NAG, col = e % NAG;
    double la = 0.0, lg = 0.0;
    if (col < 4 * R) {
      const int grp = col / R, k = col % R;
      if (grp == 0) la = lrow(g, d, a, k, SP_PIA, 1.0, -1, 0.0);
      else if (grp == 1) la = lrow(g, d, a, k, SP_PIB, 1.0, -1, 0.0);
      else if (grp == 2) la = lrow(g, d, a, k, -1, 0.0, SD_WRS, 1.0);
      else la = lrow(g, d, a, k, -1, 0.0, SD_VB, 1.0);
    } else if (col < JL) {
      la = (col - 4 * R == a && a < nPi) ? 1.0 : 0.0;
    } else if (col < JL + 2 * R) {
      const int grp = (col - JL) / R, k = (col - JL) % R;
      lg = grp == 0 ? lrow(g, d, a, k, -1, 0.0, SD_BB, 1.0) : lrow(g, d, a, k, SP_PIE, 1.0, -1, 0.0);
    } else if (col < JL + JP) {
      lg = (col - JL - 2 * R == a && a < nPi) ? 1.0 : 0.0;
    } else {
      const int k = col - JL - JP;
      la = lrow(g, d, a, k, SP_DPIB, -1.0, SD_VB, -1.0);
      lg = lrow(g, d, a, k, SP_PPIB, 1.0, SD_BB, 1.0);
    }
    db[q.LA + (long long)a * NAG + col] = la;
    db[q.LG + (long long)a * NAG + col] = lg;
  }
  // Ac[, 0:R] = y-bar = c-hat ; the copies of y in RAG and RK
  for (int e = threadIdx.x; e < M * R; e += blockDim.x) {
    const int j = e / R, k = e % R;
    const double ch = db[d.oC + e], y = db[d.oY + e];
    db[q.Ac + (long long)j * Jc + k] = ch;
    db[q.ybar + e] = ch;
    db[q.RAG + (long long)j * NAG + JL + JP + k] = y;
    db[q.RK + (long long)j * NK + 2 * Jc + R + k] = y;
  }
  __syncthreads();  // Bc is read below
  // LK: Uc starts as E_Gamma Bc, fr as the data f (zero on the interface rows)
  const int nIB = d.nI + d.nB;
  for (int e = threadIdx.x; e < m * Jc; e += blockDim.x) {
    const int r = e / Jc, col = e % Jc;
    db[q.LK + (long long)r * NK + col] = r >= m - nG ? db[q.Bc + (long long)(r - (m - nG)) * Jc + col] : 0.0;
  }
  for (int e = threadIdx.x; e < m * R; e += blockDim.x) {
    const int r = e / R, k = e % R;
    db[q.LK + (long long)r * NK + 2 * Jc + k] = r < nIB ? db[d.oF + (long long)r * R + k] : 0.0;
  }
  // PF = [pv_s - pv_r | pv-bar], WF = [theta w-bar | v_s - v_r] on the Delta rows
  for (int e = threadIdx.x; e < nDl * JF; e += blockDim.x) {
    const int r = e / JF, col = e % JF, k = col % R, a = nPi + r;
    double pf, wf;
    if (col < R) {
      pf = lrow(g, d, a, k, -1, 0.0, SD_PVSR, 1.0);
      wf = lrow(g, d, a, k, -1, 0.0, SD_WB, g.theta);
    } else {
      pf = lrow(g, d, a, k, -1, 0.0, SD_PVB, 1.0);
      wf = lrow(g, d, a, k, -1, 0.0, SD_VSR, 1.0);
    }
    db[q.PF + e] = pf;
    db[q.WFm + e] = wf;
  }
  __syncthreads();  // WF is read below
  // LKb: Ub starts as E_Delta WF
  for (int e = threadIdx.x; e < m * JF; e += blockDim.x) {
    const int r = e / JF, col = e % JF;
    db[q.LKb + (long long)r * 2 * JF + col] = r >= m - nDl ? db[q.WFm + (long long)(r - (m - nDl)) * JF + col] : 0.0;
  }
}

// One block per descriptor: a fixed-order block reduction (bitwise reproducible).
__global__ void __launch_bounds__(256) scale_dot_kernel(const DotDesc *__restrict__ dots, const double *__restrict__ db,
                                                        double *__restrict__ out) {
  __shared__ double red[256];
  const DotDesc dd = dots[blockIdx.x];
  double acc = 0.0;
  const long long n = (long long)dd.rows * dd.cols;
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const long long r = e / dd.cols, col = e % dd.cols;
    acc = fma(db[dd.a + r * dd.lda + col], db[dd.b + r * dd.ldb + col], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Per subdomain (descriptors of a subdomain are contiguous), then the total.
__global__ void __launch_bounds__(256) scale_total_kernel(const DotDesc *__restrict__ dots, int n_dots,
                                                          const SubDev *__restrict__ subs, int n_sub, double eps_rel,
                                                          double *__restrict__ gs) {
  __shared__ double red[256];
  for (int i = threadIdx.x; i < n_sub; i += blockDim.x) gs[n_dots + i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < n_sub; ++i) {
      double lin = 0.0, e2k = 0.0, kdk = 0.0, e2b = 0.0, kbdkb = 0.0;
      while (k < n_dots && dots[k].sub == i) {
        const double v = dots[k].coef * gs[k];
        switch (dots[k].role) {
          case DOT_LIN: lin += v; break;
          case DOT_E2K: e2k += v; break;
          case DOT_KDK: kdk += v; break;
          case DOT_E2KB: e2b += v; break;
          default: kbdkb += v; break;
        }
        ++k;
      }
      const double f = 2.0 * eps_rel * eps_rel / double(subs[i].M);
      gs[n_dots + i] = lin + f * e2k * kdk + f * e2b * kbdkb;
    }
  }
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < n_sub; i += blockDim.x) acc += gs[n_dots + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) gs[n_dots + n_sub] = red[0];
}

}  // namespace

cudaError_t launch_scale_gather(const Plan &p, void *ws, int wave, double theta, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  GatherArgs g;
  g.subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  g.sc = reinterpret_cast<const ScaleSub *>(base + p.off_scsub);
  g.ints = reinterpret_cast<const int *>(base + p.off_ints);
  g.db = reinterpret_cast<double *>(base + p.off_dbl);
  g.sub0 = wave * p.wave;
  g.R = p.n_rhs;
  g.n_pi = p.n_pi;
  g.n_dl = p.n_dl;
  g.JL = p.sc_JL;
  g.JP = p.sc_JP;
  g.JF = p.sc_JF;
  g.Jc = p.sc_Jc;
  g.NK = p.sc_NK;
  g.NAG = p.sc_NAG;
  g.bkd = p.o_bank_dl;
  g.bkp = p.o_bank_pi;
  g.Db = p.o_cDb;
  g.SPb = p.o_cSPb;
  g.theta = theta;
  const int n = std::min(p.n_sub, g.sub0 + p.wave) - g.sub0;
  if (n <= 0) return cudaSuccess;
  { scale_gather_kernel<<<n, 256, 0, s>>>(g); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_scale_dots(const Plan &p, void *ws, int wave, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const DotDesc *dots = reinterpret_cast<const DotDesc *>(base + p.off_dots);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  const int d0 = p.wave_dot0[wave], d1 = p.wave_dot0[wave + 1];
  if (d1 <= d0) return cudaSuccess;
  { scale_dot_kernel<<<d1 - d0, 256, 0, s>>>(dots + d0, db, db + p.o_gs + d0); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_scale_total(const Plan &p, void *ws, double eps_rel, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const DotDesc *dots = reinterpret_cast<const DotDesc *>(base + p.off_dots);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  { scale_total_kernel<<<1, 256, 0, s>>>(dots, int(p.dots.size()), subs, p.n_sub, eps_rel, db + p.o_gs); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

}  // namespace ddelm
