// Persistent interface solve: right-hand side of Eq. (nn-mixed), CG on
// Eq. (nn-mixed) (plain CG from mu = 0, stopped on the relative residual,
// Sec. 4), and the reconstruction [c; mu_Pi] = K~^+ (f~ - B~ mu_Delta) of
// Eq. (coarse_sol_2) -- one cooperative launch, one CTA per SM.
//
// The operator S_theta = B~^T (I - K~ K~^+) B~ + D~^T W D~ with
// W = theta P^T P + (1 - theta) I is applied through the local operators
//   Lambda^i = A_m^i K^+ E_Gamma   (D_ab = sum_i R_a^T Lambda^i R_b, Sec. 3),
//   Psi^i    = E_Gamma^T K K^+ E_Gamma (B^T K K^+ B = sum_i R^T Psi^i R),
//   Phi^i    = A-bar^i K-bar^+ E_Delta (P = -sum_i R_f^T Phi^i R_f, Sec. 3.1),
// and the factored coarse matrix S_Pi (Sec. 3; the application of K~^+ and of
// (K~^+)^T on [phi; 0] reduce to S_Pi^{-1} and the blocks above).  Interface
// sums are gathers over the fixed owner lists of every Pi / Delta point, so
// every run is bitwise reproducible.  All grid barriers are bounded: a barrier
// that waits too long sets the error word and every CTA returns.
#include <cooperative_groups.h>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

constexpr int CG_THREADS = 512;
constexpr int CG_WARPS = CG_THREADS / 32;

// Δ vectors ([n_dl x R]) and Π vectors ([n_pi x R]) inside the CG region
enum DlVec { V_MU = 0, V_RES, V_PD, V_Q, V_V, V_BKB, V_PV, V_W, V_B, V_TMP, N_DLVEC = 12 };
enum PiVec { P_PSI = 0, P_RA, P_MPI, P_G, P_RNU, P_NU, P_DNU, P_DPI, P_PPI, P_MPF, P_GF, P_PSI2, P_S2, P_MPIF, N_PIVEC = 14 };
enum Slab { S_H1 = 0, S_H2, S_VL, S_BL, S_TL, S_T2L, S_ZL, S_YL, N_SLAB = 9 };
// inner FP32 CG (MIXED): Delta vectors, Pi vectors, local slabs
enum FDl { F_P0 = 0, F_P1, F_Q, F_R, F_D, F_SPARE, N_FDL = 6 };
enum FPv { FP_PSI = 0, FP_RA, FP_MPI, FP_G, FP_RNU, FP_NU, FP_DNU, N_FPV = 7 };
enum FSlab { FS_H1 = 0, FS_H2, FS_VL, FS_BL, FS_TL, FS_T2L, FS_VH, FS_ZL, N_FSLAB = 8 };

struct Ctx {
  const SubDev *subs;
  const int *ints;
  double *db;
  int n_sub, n_pi, n_dl, R;
  int o_pi_own, o_dl_own;
  int o_tpi, n_tpi, o_tdl, n_tdl, o_tg, n_tg, o_tc, n_tc;
  int o_dl_rows, o_gam_rows;
  long long o_Sinv, o_C1, o_C2, o_C3;
  double *dl[N_DLVEC];
  double *pv[N_PIVEC];
  double *slab[N_SLAB];
  double *red;  // [gridDim][2*16]
  unsigned *bar;  // [count, generation]
  int *err;
  unsigned long long bar_limit_ns;  // a barrier wait gives up after this long
  unsigned bar_extra;               // tests only: 1 = one arrival more than the grid (never released)
  double theta, tol;
  int max_iters;
  double *mu_out, *c_out;
  double *info;  // [0] iterations, [1..16] true residuals, [17..32] |b|, [33] refinement sweeps
  int mode;      // 0 forward solve, 1 adjoint
  // MIXED: FP32 operators and inner-CG vectors (null in FP64 precision)
  float *fb;
  long long f_Sinv, f_C1, f_C2, f_C3;
  float *fdl[N_FDL];
  float *fpv[N_FPV];
  float *fslab[N_FSLAB];
  int max_refine;
  // scale gradient (mode 4): the bank of interface vectors and the coarse cotangents
  double *bkd, *bkp;
  double *csb, *cc1b, *cc2b, *cc3b;
};

__device__ __forceinline__ double ldg_cg(const double *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Counting grid barrier with a generation word; gives up after bar_limit_ns
// of waiting (2 s unless the options set it; error word set).  The arrival is an acq_rel atomic and the wait an acquire
// load: together with the CTA barriers around them they order every thread's
// prior writes before every thread's later reads, without a full fence.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_sync(const Ctx &c) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned *count = c.bar, *gen = c.bar + 1;
    unsigned my;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(my) : "l"(gen) : "memory");
    unsigned arrived;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(count) : "memory");
    if (arrived + 1 == gridDim.x + c.bar_extra) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(count) : "memory");
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(gen), "r"(my + 1u) : "memory");
    } else {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(gen) == my) {
        if ((++spins & 1023u) == 0u) {
          if (*(volatile int *)c.err) break;
          if (global_ns() - t0 > c.bar_limit_ns) {
            atomicExch(c.err, 1);
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  return *(volatile int *)c.err == 0;
}

__device__ __forceinline__ int gwarp() { return blockIdx.x * CG_WARPS + (threadIdx.x >> 5); }
__device__ __forceinline__ int nwarps() { return gridDim.x * CG_WARPS; }
__device__ __forceinline__ int gthread() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int nthreads() { return gridDim.x * blockDim.x; }

template <int RC>
__device__ __forceinline__ void warp_sum(double (&a)[RC]) {
#pragma unroll
  for (int c = 0; c < RC; ++c)
    for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
}

// local row index of subdomain s in a slab
__device__ __forceinline__ double *slab_row(const Ctx &c, int sl, const SubDev &d, int a) {
  return c.slab[sl] + (long long)(d.loc_off + a) * c.R;
}

// ---------------------------------------------------------------- phases
// Π-row phase: H1 = Lambda_PiDelta x^, H2 = Psi_PiDelta x^ for a Δ vector x
template <int RC>
__device__ void ph_pi_rows(const Ctx &c, const double *x) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tpi; t += nwarps()) {
    const int s = c.ints[c.o_tpi + 2 * t], a = c.ints[c.o_tpi + 2 * t + 1];
    const SubDev d = c.subs[s];
    const double *lam = c.db + d.oLam + (long long)a * d.nG;
    const double *psi = c.db + d.oPsi + (long long)a * d.nG;
    const int *gdl = c.ints + d.gdl_off;
    double h1[RC], h2[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) h1[k] = h2[k] = 0.0;
    for (int b = lane; b < d.nDl; b += 32) {
      const double la = lam[d.nPi + b], ps = psi[d.nPi + b];
      const double *xv = x + (long long)gdl[b] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) {
          const double xx = ldg_cg(xv + k);
          h1[k] = fma(la, xx, h1[k]);
          h2[k] = fma(ps, xx, h2[k]);
        }
    }
    warp_sum<RC>(h1);
    warp_sum<RC>(h2);
    if (lane == 0) {
      double *o1 = slab_row(c, S_H1, d, a), *o2 = slab_row(c, S_H2, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) {
          o1[k] = h1[k];
          o2[k] = h2[k];
        }
    }
  }
}

// Π gather: out1[π] = s1 * sum_owners slab1, out2[π] = s2 * sum_owners slab2
__device__ void ph_pi_gather(const Ctx &c, int sl1, double s1, double *out1, int sl2, double s2,
                             double *out2) {
  for (int e = gthread(); e < c.n_pi * c.R; e += nthreads()) {
    const int p = e / c.R, k = e % c.R;
    double a1 = 0.0, a2 = 0.0;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      a1 += ldg_cg(slab_row(c, sl1, d, a) + k);
      if (out2) a2 += ldg_cg(slab_row(c, sl2, d, a) + k);
    }
    out1[e] = s1 * a1;
    if (out2) out2[e] = s2 * a2;
  }
}

// coarse dense products: o1 = A1 x1 + B1 y1, o2 = A2 x2 + B2 y2 (B*, o2 optional)
__device__ void ph_coarse(const Ctx &c, long long A1, const double *x1, long long B1, const double *y1,
                          double b1s, double *o1, long long A2, const double *x2, long long B2,
                          const double *y2, double b2s, double *o2) {
  const int lane = threadIdx.x & 31;
  const int n = c.n_pi;
  for (int t = gwarp(); t < n * c.R; t += nwarps()) {
    const int p = t / c.R, k = t % c.R;
    double s1 = 0.0, s2 = 0.0;
    for (int q = lane; q < n; q += 32) {
      const long long e = (long long)p * n + q;
      s1 = fma(c.db[A1 + e], ldg_cg(x1 + (long long)q * c.R + k), s1);
      if (B1 >= 0) s1 = fma(b1s * c.db[B1 + e], ldg_cg(y1 + (long long)q * c.R + k), s1);
      if (o2) {
        s2 = fma(c.db[A2 + e], ldg_cg(x2 + (long long)q * c.R + k), s2);
        if (B2 >= 0) s2 = fma(b2s * c.db[B2 + e], ldg_cg(y2 + (long long)q * c.R + k), s2);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      o1[t] = s1;
      if (o2) o2[t] = s2;
    }
  }
}

// Δ-row phase of the first half of S_theta (and of b_theta):
//   lambda = [R_Pi piv; lsign * R_Delta x]  (piv: Π vector, x: Δ vector or null)
//   VL = -(Lambda lambda + addA)_Delta ; BL = bsign*(lambda - Psi lambda)_Delta + addP + Lambda_PiD^T g
// RHS mode (rhs=1): VL = -(a + Lambda lambda)_Δ, BL = (p + Psi lambda)_Δ + Lambda_PiD^T g
template <int RC>
__device__ void ph_dl_first(const Ctx &c, const double *piv, const double *x, const double *g, int rhs) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tdl; t += nwarps()) {
    const int s = c.ints[c.o_tdl + 2 * t], dd = c.ints[c.o_tdl + 2 * t + 1];
    const SubDev d = c.subs[s];
    const int a = d.nPi + dd;
    const double *lam = c.db + d.oLam + (long long)a * d.nG;
    const double *psi = c.db + d.oPsi + (long long)a * d.nG;
    const double *lamT = c.db + d.oLamT + (long long)a * d.nG;
    const int *gpi = c.ints + d.gpi_off;
    const int *gdl = c.ints + d.gdl_off;
    double sl[RC], sp[RC], sg[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) sl[k] = sp[k] = sg[k] = 0.0;
    const int bmax = rhs ? d.nPi : d.nG;
    for (int b = lane; b < bmax; b += 32) {
      const double la = lam[b], ps = psi[b];
      const double *src;
      double sgn;
      if (b < d.nPi) {
        src = piv + (long long)gpi[b] * c.R;
        sgn = 1.0;
      } else {
        src = x + (long long)gdl[b - d.nPi] * c.R;
        sgn = -1.0;
      }
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) {
          const double v = sgn * ldg_cg(src + k);
          sl[k] = fma(la, v, sl[k]);
          sp[k] = fma(ps, v, sp[k]);
        }
    }
    for (int b = lane; b < d.nPi; b += 32) {
      const double lt = lamT[b];
      const double *src = g + (long long)gpi[b] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) sg[k] = fma(lt, ldg_cg(src + k), sg[k]);
    }
    warp_sum<RC>(sl);
    warp_sum<RC>(sp);
    warp_sum<RC>(sg);
    if (lane == 0) {
      double *vo = slab_row(c, S_VL, d, a), *bo = slab_row(c, S_BL, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) {
          if (rhs) {
            const double av = c.db[d.oAy + (long long)a * c.R + k];
            const double pv = c.db[d.oP + (long long)a * c.R + k];
            vo[k] = -(av + sl[k]);
            bo[k] = pv + sp[k] + sg[k];
          } else {
            const double lama = -ldg_cg(x + (long long)gdl[dd] * c.R + k);
            vo[k] = -sl[k];
            bo[k] = -(lama - sp[k]) + sg[k];
          }
        }
    }
  }
}

// sum of a slab column over the owners of Δ point p: two, or four for the
// cross points of vanilla DDELM (rows -1 past the owners)
__device__ __forceinline__ double dl_owner_sum(const Ctx &c, const double *slab, int p, int k) {
  const int4 rw = *reinterpret_cast<const int4 *>(c.ints + c.o_dl_rows + 4 * p);
  double v = ldg_cg(slab + (long long)rw.x * c.R + k) + ldg_cg(slab + (long long)rw.y * c.R + k);
  if (rw.z >= 0) v += ldg_cg(slab + (long long)rw.z * c.R + k) + ldg_cg(slab + (long long)rw.w * c.R + k);
  return v;
}

// Δ gather: out[δ] = s * (sum of slab over the owners) + t * add[δ]
__device__ void ph_dl_gather(const Ctx &c, int sl, double s, double *out, const double *add, double t,
                             int sl2, double *out2) {
  for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) {
    const int p = e / c.R, k = e % c.R;
    double r = s * dl_owner_sum(c, c.slab[sl], p, k);
    if (add) r = fma(t, ldg_cg(add + e), r);
    out[e] = r;
    if (out2) out2[e] = dl_owner_sum(c, c.slab[sl2], p, k);
  }
}

// Δ-row local products with Phi or Phi^T: slab[nPi + d] = -sum_e M[d][e] x[gdl[e]]
template <int RC>
__device__ void ph_dl_phi(const Ctx &c, bool transposed, const double *x, int sl) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tdl; t += nwarps()) {
    const int s = c.ints[c.o_tdl + 2 * t], dd = c.ints[c.o_tdl + 2 * t + 1];
    const SubDev d = c.subs[s];
    const double *row = c.db + (transposed ? d.oPhiT : d.oPhi) + (long long)dd * d.nDl;
    const int *gdl = c.ints + d.gdl_off;
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int e = lane; e < d.nDl; e += 32) {
      const double m = row[e];
      const double *src = x + (long long)gdl[e] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(m, ldg_cg(src + k), acc[k]);
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
      double *o = slab_row(c, sl, d, d.nPi + dd);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) o[k] = -acc[k];
    }
  }
}

// Γ-row phase: ZL = Lambda^T [0; w^]  (all nG rows)
template <int RC>
__device__ void ph_g_lamT(const Ctx &c, const double *w) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tg; t += nwarps()) {
    const int s = c.ints[c.o_tg + 2 * t], a = c.ints[c.o_tg + 2 * t + 1];
    const SubDev d = c.subs[s];
    const double *row = c.db + d.oLamT + (long long)a * d.nG;
    const int *gdl = c.ints + d.gdl_off;
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int e = lane; e < d.nDl; e += 32) {
      const double m = row[d.nPi + e];
      const double *src = w + (long long)gdl[e] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(m, ldg_cg(src + k), acc[k]);
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
      double *o = slab_row(c, S_ZL, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) o[k] = acc[k];
    }
  }
}

// Δ-row phase: YL = ZL_Delta + Psi_DeltaPi nu^ - Lambda_PiDelta^T Dnu^
template <int RC>
__device__ void ph_dl_last(const Ctx &c, const double *nu, const double *dnu, bool with_z) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tdl; t += nwarps()) {
    const int s = c.ints[c.o_tdl + 2 * t], dd = c.ints[c.o_tdl + 2 * t + 1];
    const SubDev d = c.subs[s];
    const int a = d.nPi + dd;
    const double *psi = c.db + d.oPsi + (long long)a * d.nG;
    const double *lamT = c.db + d.oLamT + (long long)a * d.nG;
    const int *gpi = c.ints + d.gpi_off;
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int b = lane; b < d.nPi; b += 32) {
      const double ps = psi[b], lt = lamT[b];
      const double *sn = nu + (long long)gpi[b] * c.R;
      const double *sd = dnu + (long long)gpi[b] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(ps, ldg_cg(sn + k), fma(-lt, ldg_cg(sd + k), acc[k]));
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
      double *o = slab_row(c, S_YL, d, a);
      const double *z = slab_row(c, S_ZL, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) o[k] = (with_z ? ldg_cg(z + k) : 0.0) + acc[k];
    }
  }
}

// block-level partial dot products of columns: red[block][k] = sum x[e][k] y[e][k].
// Walks the elements e = row*R + k with the same grid stride as the vector
// updates, so every thread reads only elements it wrote itself (no barrier is
// needed between an update loop and the dot product that follows it).
template <int RC>
__device__ void partial_dot(const Ctx &c, const double *x, const double *y, int slot) {
  __shared__ double sred[CG_WARPS][16];
  double acc[RC];
#pragma unroll
  for (int k = 0; k < RC; ++k) acc[k] = 0.0;
  const int R = c.R;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
    const double v = ldg_cg(x + e) * ldg_cg(y + e);
    const int col = e % R;
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k == col) acc[k] += v;
  }
  warp_sum<RC>(acc);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < RC; ++k) sred[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < RC) {
    double s = 0.0;
    for (int w = 0; w < CG_WARPS; ++w) s += sred[w][threadIdx.x];
    c.red[(long long)blockIdx.x * 32 + slot * 16 + threadIdx.x] = s;
  }
  __syncthreads();
}

// every CTA sums the partials in the same order: out[k] (shared)
template <int RC>
__device__ void finish_dot(const Ctx &c, int slot, double *out) {
  if (threadIdx.x < RC) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ldg_cg(c.red + (long long)b * 32 + slot * 16 + threadIdx.x);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// From the VL/BL slabs: v = sum VL (= D~ x), bkb = sum BL, and w = W v with
// W = theta P^T P + (1 - theta) I.
template <int RC>
__device__ bool apply_W(const Ctx &c) {
  double *v = c.dl[V_V], *bkb = c.dl[V_BKB], *pvv = c.dl[V_PV], *w = c.dl[V_W];
  ph_dl_gather(c, S_VL, 1.0, v, nullptr, 0.0, S_BL, bkb);  // v = D~ x, bkb
  if (!grid_sync(c)) return false;
  ph_dl_phi<RC>(c, false, v, S_TL);  // -Phi v^
  if (!grid_sync(c)) return false;
  ph_dl_gather(c, S_TL, 1.0, pvv, nullptr, 0.0, -1, nullptr);  // P v
  if (!grid_sync(c)) return false;
  ph_dl_phi<RC>(c, true, pvv, S_T2L);  // -Phi^T (P v)^
  if (!grid_sync(c)) return false;
  ph_dl_gather(c, S_T2L, c.theta, w, v, 1.0 - c.theta, -1, nullptr);  // W v
  return grid_sync(c);
}

// Second half of the operator: given VL/BL slabs (v = sum VL, bkb = sum BL),
// computes out = bkb + D~^T W v.  Returns false on a barrier timeout.
template <int RC>
__device__ bool second_half(const Ctx &c, double *out) {
  double *bkb = c.dl[V_BKB], *w = c.dl[V_W];
  if (!apply_W<RC>(c)) return false;
  ph_g_lamT<RC>(c, w);  // z = Lambda^T [0; w^]
  if (!grid_sync(c)) return false;
  ph_pi_gather(c, S_ZL, 1.0, c.pv[P_RNU], -1, 0.0, nullptr);
  if (!grid_sync(c)) return false;
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_RNU], -1, nullptr, 0.0, c.pv[P_NU], c.o_C3, c.pv[P_RNU], -1, nullptr,
              0.0, c.pv[P_DNU]);
  if (!grid_sync(c)) return false;
  ph_dl_last<RC>(c, c.pv[P_NU], c.pv[P_DNU], true);
  if (!grid_sync(c)) return false;
  ph_dl_gather(c, S_YL, 1.0, out, bkb, 1.0, -1, nullptr);
  return grid_sync(c);
}

// q = S_theta x for a Δ vector x
template <int RC>
__device__ bool apply_S(const Ctx &c, const double *x, double *q) {
  ph_pi_rows<RC>(c, x);
  if (!grid_sync(c)) return false;
  ph_pi_gather(c, S_H1, 1.0, c.pv[P_PSI], S_H2, -1.0, c.pv[P_RA]);
  if (!grid_sync(c)) return false;
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_RA], c.o_C1, c.pv[P_PSI], 1.0, c.pv[P_MPI], c.o_C2, c.pv[P_PSI], c.o_C3,
              c.pv[P_RA], -1.0, c.pv[P_G]);
  if (!grid_sync(c)) return false;
  ph_dl_first<RC>(c, c.pv[P_MPI], x, c.pv[P_G], 0);
  if (!grid_sync(c)) return false;
  return second_half<RC>(c, q);
}

// Plain CG on S_theta mu = B from mu = 0 (per right-hand side, converged
// columns frozen); returns the iteration count or -1 on a barrier timeout.
// s_bn receives |B| per column.
template <int RC>
__device__ int cg_solve(const Ctx &c, double *s_bn) {
  __shared__ double s_rr[16], s_pq[16], s_rn[16], s_alpha[16], s_beta[16];
  __shared__ int s_done;
  double *B = c.dl[V_B], *MU = c.dl[V_MU], *RES = c.dl[V_RES], *PD = c.dl[V_PD], *Q = c.dl[V_Q];
  for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) {
    const double b = B[e];
    MU[e] = 0.0;
    RES[e] = b;
    PD[e] = b;
  }
  partial_dot<RC>(c, B, B, 0);
  if (!grid_sync(c)) return -1;
  finish_dot<RC>(c, 0, s_bn);
  if (threadIdx.x < RC) {
    s_rr[threadIdx.x] = s_bn[threadIdx.x];
    s_bn[threadIdx.x] = sqrt(s_bn[threadIdx.x]);
  }
  if (threadIdx.x == 0) s_done = 0;
  __syncthreads();
  int it = 0;
  while (true) {
    if (threadIdx.x == 0) {
      int done = 1;
      for (int k = 0; k < c.R && k < RC; ++k)
        if (s_bn[k] > 0.0 && sqrt(s_rr[k]) >= c.tol * s_bn[k]) done = 0;
      s_done = done || it >= c.max_iters;
    }
    __syncthreads();
    if (s_done) break;
    if (!apply_S<RC>(c, PD, Q)) return -1;
    partial_dot<RC>(c, PD, Q, 0);
    if (!grid_sync(c)) return -1;
    finish_dot<RC>(c, 0, s_pq);
    if (threadIdx.x < RC) {
      const int k = threadIdx.x;
      const bool live = k < c.R && s_bn[k] > 0.0 && sqrt(s_rr[k]) >= c.tol * s_bn[k] && s_pq[k] != 0.0;
      s_alpha[k] = live ? s_rr[k] / s_pq[k] : 0.0;
    }
    __syncthreads();
    for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) {
      const double al = s_alpha[e % c.R];
      MU[e] = fma(al, PD[e], MU[e]);
      RES[e] = fma(-al, ldg_cg(Q + e), RES[e]);
    }
    partial_dot<RC>(c, RES, RES, 1);
    if (!grid_sync(c)) return -1;
    finish_dot<RC>(c, 1, s_rn);
    if (threadIdx.x < RC) {
      const int k = threadIdx.x;
      s_beta[k] = (s_alpha[k] != 0.0 && s_rr[k] > 0.0) ? s_rn[k] / s_rr[k] : 0.0;
      if (s_alpha[k] != 0.0) s_rr[k] = s_rn[k];
    }
    __syncthreads();
    for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) {
      const double be = s_beta[e % c.R];
      if (s_alpha[e % c.R] != 0.0) PD[e] = fma(be, PD[e], RES[e]);
    }
    ++it;
    if (!grid_sync(c)) return -1;
  }
  return it;
}

// ================================================================ MIXED
// Inner FP32 CG on S_theta (the FP32 copies of Lambda, Lambda^T, Psi, Phi,
// Phi^T and of the coarse matrices), organised per subdomain: a CTA stages the
// subdomain's local vector (gathered from the owners' slab rows) in shared
// memory and its warps take the rows of the local operator, so that the
// interface gathers cost no extra phase.  FP64 iterative refinement around it
// (residuals of the FP64 operator) recovers the FP64 solution.

constexpr int MAXG = 256;   // largest local interface (nG) staged in shared memory

// the staged local vector [nG][R] (then 64 floats of Pi-row data); one buffer
// for every per-subdomain phase (they never overlap within a CTA)
__shared__ float sh_stage[MAXG * 16 + 64];

__device__ __forceinline__ float *fslab_row(const Ctx &c, int sl, const SubDev &d, int a) {
  return c.fslab[sl] + (long long)(d.loc_off + a) * c.R;
}

// Row product with a shared-memory vector: sum_j m[j] xs[j*R + k].  RC == 1:
// lanes over j, the result in every lane; RC == 16: lane = k + 16 h takes the
// j of parity h, the result for column k in lanes k and k + 16.
template <int RC>
__device__ __forceinline__ float row_dot(const float *__restrict__ m, int n, const float *xs, int R) {
  const int lane = threadIdx.x & 31;
  float a = 0.f;
  if (RC == 1) {
    for (int j = lane; j < n; j += 32) a = fmaf(__ldg(m + j), xs[j], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  } else {
    const int k = lane & 15, h = lane >> 4;
    for (int j0 = 0; j0 < n; j0 += 32) {
      const float mv = (j0 + lane < n) ? __ldg(m + j0 + lane) : 0.f;
#pragma unroll 4
      for (int jj = 0; jj < 32; jj += 2) {
        const float mm = __shfl_sync(0xffffffffu, mv, jj + h);
        const int j = j0 + jj + h;
        if (j < n && k < R) a = fmaf(mm, xs[j * R + k], a);
      }
    }
    a += __shfl_xor_sync(0xffffffffu, a, 16);
  }
  return a;
}

// cnt <= 4 consecutive rows (stride ld) at once, so that their loads overlap
template <int RC>
__device__ __forceinline__ void row_dot4(const float *__restrict__ m, long long ld, int cnt, int n, const float *xs,
                                         int R, float (&v)[4]) {
  if (RC == 1) {
    const int lane = threadIdx.x & 31;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = lane; j < n; j += 32) {
      const float x = xs[j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < cnt) a[i] = fmaf(__ldg(m + i * ld + j), x, a[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
      v[i] = a[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = i < cnt ? row_dot<RC>(m + i * ld, n, xs, R) : 0.f;
  }
}

// the lane that stores column k of a row_dot result (k < R)
template <int RC>
__device__ __forceinline__ bool row_writer(int R, int &k) {
  const int lane = threadIdx.x & 31;
  if (RC == 1) {
    k = 0;
    return lane == 0;
  }
  k = lane;
  return lane < R;
}

// work items of a per-subdomain phase: (subdomain, row chunk)
__device__ __forceinline__ int n_chunks(const Ctx &c) {
  int ch = (int)gridDim.x / c.n_sub;  // at most one work item per CTA
  return ch < 1 ? 1 : (ch > 8 ? 8 : ch);
}

// gathered slab sum at the Delta point of local interface row (d, a): its
// owners' rows (two, or four for a cross point of vanilla DDELM), column k
__device__ __forceinline__ float gam_pair(const Ctx &c, int sl, const SubDev &d, int a, int k) {
  const int4 rw = *reinterpret_cast<const int4 *>(c.ints + c.o_gam_rows + 4 * (d.loc_off + a));
  float v = __ldcg(c.fslab[sl] + (long long)rw.x * c.R + k) + __ldcg(c.fslab[sl] + (long long)rw.y * c.R + k);
  if (rw.z >= 0) v += __ldcg(c.fslab[sl] + (long long)rw.z * c.R + k) + __ldcg(c.fslab[sl] + (long long)rw.w * c.R + k);
  return v;
}

// The vector S is applied to: x itself (xp == nullptr), or the CG direction
// The direction p_i = (r_{i-1} - a q_{i-1}) + b p_{i-1} formed on the fly from
// vectors completed before the previous reduction (a = alpha_{i-1}, b =
// beta_{i-1} per column; absent terms: null), bit for bit what the owners'
// update stores, so that no grid barrier separates that update from the
// next application.
struct DirIn {
  const float *r, *q, *p;
  const float *a, *b;  // per column, shared memory
};
__device__ __forceinline__ float dir_at(const DirIn &v, long long idx, int k) {
  float x = __ldcg(v.r + idx);
  if (v.q) x = fmaf(-v.a[k], __ldcg(v.q + idx), x);
  if (v.p) x = fmaf(v.b[k], __ldcg(v.p + idx), x);
  return x;
}

// P1: H1 = Lambda_{Pi,Delta} x^, H2 = Psi_{Pi,Delta} x^ (the few Pi rows)
template <int RC>
__device__ void f_pi_rows(const Ctx &c, const DirIn &x) {
  float *xs = sh_stage;
  const int R = c.R, w = threadIdx.x >> 5;
  for (int s = blockIdx.x; s < c.n_sub; s += gridDim.x) {
    const SubDev d = c.subs[s];
    if (d.nPi == 0) continue;
    const int *gdl = c.ints + d.gdl_off;
    for (int e = threadIdx.x; e < d.nDl * R; e += blockDim.x) xs[e] = dir_at(x, (long long)gdl[e / R] * R + e % R, e % R);
    __syncthreads();
    const float *lam = c.fb + d.oLam32, *psi = c.fb + d.oPsi32;
    for (int t = w; t < 2 * d.nPi; t += CG_WARPS) {
      const int a = t >> 1;
      const float *row = ((t & 1) ? psi : lam) + (long long)a * d.nG + d.nPi;
      const float v = row_dot<RC>(row, d.nDl, xs, R);
      int k;
      if (row_writer<RC>(R, k)) fslab_row(c, (t & 1) ? FS_H2 : FS_H1, d, a)[k] = v;
    }
    __syncthreads();
  }
}

// Pi gathers: out1 = s1 sum slab1, out2 = s2 sum slab2
__device__ void f_pi_gather(const Ctx &c, int sl1, float s1, float *out1, int sl2, float s2, float *out2) {
  for (int e = gthread(); e < c.n_pi * c.R; e += nthreads()) {
    const int p = e / c.R, k = e % c.R;
    float a1 = 0.f, a2 = 0.f;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      a1 += __ldcg(fslab_row(c, sl1, d, a) + k);
      if (out2) a2 += __ldcg(fslab_row(c, sl2, d, a) + k);
    }
    out1[e] = s1 * a1;
    if (out2) out2[e] = s2 * a2;
  }
}

// coarse products: o1 = A1 x1 + b1s B1 y1, o2 = A2 x2 + b2s B2 y2 (FP32 matrices; B*, o2 optional)
__device__ void f_coarse(const Ctx &c, long long A1, const float *x1, long long B1, const float *y1, float b1s,
                         float *o1, long long A2, const float *x2, long long B2, const float *y2, float b2s,
                         float *o2) {
  const int lane = threadIdx.x & 31;
  const int n = c.n_pi, R = c.R;
  for (int t = gwarp(); t < n * R; t += nwarps()) {
    const int p = t / R, k = t % R;
    float s1 = 0.f, s2 = 0.f;
    for (int q = lane; q < n; q += 32) {
      const long long e = (long long)p * n + q;
      s1 = fmaf(c.fb[A1 + e], __ldcg(x1 + q * R + k), s1);
      if (B1 >= 0) s1 = fmaf(b1s * c.fb[B1 + e], __ldcg(y1 + q * R + k), s1);
      if (o2) {
        s2 = fmaf(c.fb[A2 + e], __ldcg(x2 + q * R + k), s2);
        if (B2 >= 0) s2 = fmaf(b2s * c.fb[B2 + e], __ldcg(y2 + q * R + k), s2);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      o1[t] = s1;
      if (o2) o2[t] = s2;
    }
  }
}

// P3: lambda = [R_Pi mpi; -x^]; VL = -(Lambda lambda)_Delta ;
//     BL = -(lambda - Psi lambda)_Delta + Lambda_{Pi,Delta}^T g_Pi
template <int RC>
__device__ void f_dl_first(const Ctx &c, const DirIn &x, const float *mpi, const float *g) {
  float *xs = sh_stage, *gs = sh_stage + MAXG * 16;
  const int R = c.R, w = threadIdx.x >> 5;
  const int ch = n_chunks(c);
  for (int it = blockIdx.x; it < c.n_sub * ch; it += gridDim.x) {
    const int s = it / ch, q = it % ch;
    const SubDev d = c.subs[s];
    const int r0 = (d.nDl * q) / ch, r1 = (d.nDl * (q + 1)) / ch;
    if (r0 >= r1) continue;
    const int *gpi = c.ints + d.gpi_off, *gdl = c.ints + d.gdl_off;
    for (int e = threadIdx.x; e < d.nG * R; e += blockDim.x) {
      const int a = e / R, k = e % R;
      xs[e] = a < d.nPi ? mpi[gpi[a] * R + k] : -dir_at(x, (long long)gdl[a - d.nPi] * R + k, k);
    }
    for (int e = threadIdx.x; e < d.nPi * R; e += blockDim.x)
      gs[e] = g[gpi[e / R] * R + e % R];
    __syncthreads();
    const float *lam = c.fb + d.oLam32, *psi = c.fb + d.oPsi32, *lamT = c.fb + d.oLamT32;
    // four rows per warp at a time, so that their loads overlap
    for (int dd = r0 + 4 * w; dd < r1; dd += 4 * CG_WARPS) {
      const int cnt = min(4, r1 - dd);
      const int a0 = d.nPi + dd;
      float sl[4], sp[4], sg[4];
      row_dot4<RC>(lam + (long long)a0 * d.nG, d.nG, cnt, d.nG, xs, R, sl);
      row_dot4<RC>(psi + (long long)a0 * d.nG, d.nG, cnt, d.nG, xs, R, sp);
      row_dot4<RC>(lamT + (long long)a0 * d.nG, d.nG, cnt, d.nPi, gs, R, sg);
      int k;
      if (row_writer<RC>(R, k))
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < cnt) {
            const int a = a0 + i;
            fslab_row(c, FS_VL, d, a)[k] = -sl[i];
            fslab_row(c, FS_BL, d, a)[k] = -(xs[a * R + k] - sp[i]) + sg[i];
          }
    }
    __syncthreads();
  }
}

// P4 / P5: out = -M y^ with y^ the gathered slab `in` (M = Phi or Phi^T); P4
// also keeps v^ in the VH slab
template <int RC>
__device__ void f_dl_phi(const Ctx &c, bool transposed, int in, int out, bool keep_v) {
  float *xs = sh_stage;
  const int R = c.R, w = threadIdx.x >> 5;
  const int ch = n_chunks(c);
  for (int it = blockIdx.x; it < c.n_sub * ch; it += gridDim.x) {
    const int s = it / ch, q = it % ch;
    const SubDev d = c.subs[s];
    const int r0 = (d.nDl * q) / ch, r1 = (d.nDl * (q + 1)) / ch;
    if (r0 >= r1) continue;
    for (int e = threadIdx.x; e < d.nDl * R; e += blockDim.x) {
      const int b = e / R, k = e % R;
      const float v = gam_pair(c, in, d, d.nPi + b, k);
      xs[e] = v;
      if (keep_v && b >= r0 && b < r1) fslab_row(c, FS_VH, d, d.nPi + b)[k] = v;
    }
    __syncthreads();
    const float *M = c.fb + (transposed ? d.oPhiT32 : d.oPhi32);
    for (int dd = r0 + 4 * w; dd < r1; dd += 4 * CG_WARPS) {
      const int cnt = min(4, r1 - dd);
      float v[4];
      row_dot4<RC>(M + (long long)dd * d.nDl, d.nDl, cnt, d.nDl, xs, R, v);
      int k;
      if (row_writer<RC>(R, k))
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < cnt) fslab_row(c, out, d, d.nPi + dd + i)[k] = -v[i];
    }
    __syncthreads();
  }
}

// P6: w^ = theta (sum T2L)^ + (1 - theta) v^ ; ZL = Lambda^T [0; w^] (all Gamma rows)
template <int RC>
__device__ void f_g_lamT(const Ctx &c) {
  float *xs = sh_stage;
  const int R = c.R, w = threadIdx.x >> 5;
  const int ch = n_chunks(c);
  const float th = (float)c.theta;
  for (int it = blockIdx.x; it < c.n_sub * ch; it += gridDim.x) {
    const int s = it / ch, q = it % ch;
    const SubDev d = c.subs[s];
    const int r0 = (d.nG * q) / ch, r1 = (d.nG * (q + 1)) / ch;
    if (r0 >= r1) continue;
    for (int e = threadIdx.x; e < d.nDl * R; e += blockDim.x) {
      const int b = e / R, k = e % R;
      xs[e] = th * gam_pair(c, FS_T2L, d, d.nPi + b, k) + (1.f - th) * __ldcg(fslab_row(c, FS_VH, d, d.nPi + b) + k);
    }
    __syncthreads();
    const float *lamT = c.fb + d.oLamT32;
    for (int a = r0 + 4 * w; a < r1; a += 4 * CG_WARPS) {
      const int cnt = min(4, r1 - a);
      float v[4];
      row_dot4<RC>(lamT + (long long)a * d.nG + d.nPi, d.nG, cnt, d.nDl, xs, R, v);
      int k;
      if (row_writer<RC>(R, k))
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (i < cnt) fslab_row(c, FS_ZL, d, a + i)[k] = v[i];
    }
    __syncthreads();
  }
}

// YL of local Delta row a (column k): ZL + Psi_{Delta,Pi} nu^ - Lambda_{Pi,Delta}^T Dnu^
__device__ __forceinline__ float f_yl(const Ctx &c, const SubDev &d, int a, int k, const float *nu,
                                     const float *dnu) {
  const int *gpi = c.ints + d.gpi_off;
  const float *psi = c.fb + d.oPsi32 + (long long)a * d.nG;
  const float *lamT = c.fb + d.oLamT32 + (long long)a * d.nG;
  float v = __ldcg(fslab_row(c, FS_ZL, d, a) + k);
  for (int b = 0; b < d.nPi; ++b) {
    const int gp = gpi[b];
    v = fmaf(psi[b], nu[gp * c.R + k], v);
    v = fmaf(-lamT[b], dnu[gp * c.R + k], v);
  }
  return v;
}

// Small coarse spaces (|Pi|^2 R <= 4096): every CTA gathers the Pi sums and
// applies the coarse matrices itself, in shared memory, which saves the two
// grid barriers between gather and product (twice per application).
constexpr int SMALL_COARSE = 4096;
__shared__ float sh_pi[6][256];  // |Pi| R <= 256 (implied by |Pi|^2 R <= 4096, R <= 16)

__device__ __forceinline__ bool small_coarse(const Ctx &c) {
  return c.n_pi > 0 && c.n_pi * c.n_pi * c.R <= SMALL_COARSE;
}

// in shared memory: o1 = s1 sum sl1 over the Pi owners, o2 = s2 sum sl2 (o2 optional)
__device__ void f_pi_gather_local(const Ctx &c, int sl1, float s1, float *o1, int sl2, float s2, float *o2) {
  for (int e = threadIdx.x; e < c.n_pi * c.R; e += blockDim.x) {
    const int p = e / c.R, k = e % c.R;
    float a1 = 0.f, a2 = 0.f;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      a1 += __ldcg(fslab_row(c, sl1, d, a) + k);
      if (o2) a2 += __ldcg(fslab_row(c, sl2, d, a) + k);
    }
    o1[e] = s1 * a1;
    if (o2) o2[e] = s2 * a2;
  }
}

// in shared memory: o1 = A1 x1 + b1s B1 y1, o2 = A2 x2 + b2s B2 y2 (B*, o2 optional)
__device__ void f_coarse_local(const Ctx &c, long long A1, const float *x1, long long B1, const float *y1, float b1s,
                               float *o1, long long A2, const float *x2, long long B2, const float *y2, float b2s,
                               float *o2) {
  const int n = c.n_pi, R = c.R;
  for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
    const int p = t / R, k = t % R;
    float s1 = 0.f, s2 = 0.f;
    for (int q = 0; q < n; ++q) {
      const long long e = (long long)p * n + q;
      s1 = fmaf(c.fb[A1 + e], x1[q * R + k], s1);
      if (B1 >= 0) s1 = fmaf(b1s * c.fb[B1 + e], y1[q * R + k], s1);
      if (o2) {
        s2 = fmaf(c.fb[A2 + e], x2[q * R + k], s2);
        if (B2 >= 0) s2 = fmaf(b2s * c.fb[B2 + e], y2[q * R + k], s2);
      }
    }
    o1[t] = s1;
    if (o2) o2[t] = s2;
  }
}

// q = S32 x; the last phase (gathers of YL and BL) is fused into the dot product
// p.q that follows, so this returns with q written and a partial dot pending in
// red slot 0 (no barrier taken after it).
template <int RC>
__device__ bool f_apply_S(const Ctx &c, const DirIn &x, float *q) {
  const bool sm = small_coarse(c);
  f_pi_rows<RC>(c, x);
  if (!grid_sync(c)) return false;
  const float *mpi = c.fpv[FP_MPI], *g = c.fpv[FP_G];
  if (sm) {
    f_pi_gather_local(c, FS_H1, 1.f, sh_pi[0], FS_H2, -1.f, sh_pi[1]);
    __syncthreads();
    f_coarse_local(c, c.f_Sinv, sh_pi[1], c.f_C1, sh_pi[0], 1.f, sh_pi[2], c.f_C2, sh_pi[0], c.f_C3, sh_pi[1], -1.f,
                   sh_pi[3]);
    __syncthreads();
    mpi = sh_pi[2];
    g = sh_pi[3];
  } else {
    f_pi_gather(c, FS_H1, 1.f, c.fpv[FP_PSI], FS_H2, -1.f, c.fpv[FP_RA]);
    if (!grid_sync(c)) return false;
    if (c.n_pi > 0)
      f_coarse(c, c.f_Sinv, c.fpv[FP_RA], c.f_C1, c.fpv[FP_PSI], 1.f, c.fpv[FP_MPI], c.f_C2, c.fpv[FP_PSI], c.f_C3,
               c.fpv[FP_RA], -1.f, c.fpv[FP_G]);
    if (!grid_sync(c)) return false;
  }
  f_dl_first<RC>(c, x, mpi, g);
  if (!grid_sync(c)) return false;
  f_dl_phi<RC>(c, false, FS_VL, FS_TL, true);
  if (!grid_sync(c)) return false;
  f_dl_phi<RC>(c, true, FS_TL, FS_T2L, false);
  if (!grid_sync(c)) return false;
  f_g_lamT<RC>(c);
  if (!grid_sync(c)) return false;
  const float *nu = c.fpv[FP_NU], *dnu = c.fpv[FP_DNU];
  if (sm) {
    f_pi_gather_local(c, FS_ZL, 1.f, sh_pi[4], -1, 0.f, nullptr);
    __syncthreads();
    f_coarse_local(c, c.f_Sinv, sh_pi[4], -1, nullptr, 0.f, sh_pi[5], c.f_C3, sh_pi[4], -1, nullptr, 0.f, sh_pi[2]);
    __syncthreads();
    nu = sh_pi[5];
    dnu = sh_pi[2];
  } else {
    f_pi_gather(c, FS_ZL, 1.f, c.fpv[FP_RNU], -1, 0.f, nullptr);
    if (!grid_sync(c)) return false;
    if (c.n_pi > 0)
      f_coarse(c, c.f_Sinv, c.fpv[FP_RNU], -1, nullptr, 0.f, c.fpv[FP_NU], c.f_C3, c.fpv[FP_RNU], -1, nullptr, 0.f,
               c.fpv[FP_DNU]);
    if (!grid_sync(c)) return false;
  }
  // q[delta] = sum_owners (YL + BL)
  for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) {
    const int gd = e / c.R, k = e % c.R;
    const int *own = c.ints + c.o_dl_own + 8 * gd;
    const SubDev &da = c.subs[own[0]];
    const SubDev &dB = c.subs[own[2]];
    const int4 rw = *reinterpret_cast<const int4 *>(c.ints + c.o_dl_rows + 4 * gd);
    float v = f_yl(c, da, da.nPi + own[1], k, nu, dnu) + f_yl(c, dB, dB.nPi + own[3], k, nu, dnu);
    if (rw.z >= 0) {  // a cross point of vanilla DDELM: four owners
      const SubDev &dc = c.subs[own[4]];
      const SubDev &dd = c.subs[own[6]];
      v += f_yl(c, dc, dc.nPi + own[5], k, nu, dnu) + f_yl(c, dd, dd.nPi + own[7], k, nu, dnu);
    }
    v = v + __ldcg(c.fslab[FS_BL] + (long long)rw.x * c.R + k);
    v = v + __ldcg(c.fslab[FS_BL] + (long long)rw.y * c.R + k);
    if (rw.z >= 0)
      v += __ldcg(c.fslab[FS_BL] + (long long)rw.z * c.R + k) + __ldcg(c.fslab[FS_BL] + (long long)rw.w * c.R + k);
    q[e] = v;
  }
  return true;
}

// partial dot of FP32 columns (FP64 accumulation past the warp level), same
// element walk as the updates
template <int RC>
__device__ void f_partial_dot(const Ctx &c, const float *x, const float *y, int slot) {
  __shared__ double sred[CG_WARPS][16];
  double acc[RC];
#pragma unroll
  for (int k = 0; k < RC; ++k) acc[k] = 0.0;
  const int R = c.R;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
    const double v = (double)__ldcg(x + e) * (double)__ldcg(y + e);
    const int col = e % R;
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k == col) acc[k] += v;
  }
  warp_sum<RC>(acc);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < RC; ++k) sred[threadIdx.x >> 5][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < RC) {
    double sm = 0.0;
    for (int w = 0; w < CG_WARPS; ++w) sm += sred[w][threadIdx.x];
    c.red[(long long)blockIdx.x * 32 + slot * 16 + threadIdx.x] = sm;
  }
  __syncthreads();
}

// The owners' step after an application q_i = S32 p_i, over the element walk
// of that application's last phase (no barrier between): r_i = r_{i-1} -
// a q_{i-1}, p_i = r_i + b p_{i-1} (the values the application formed),
// d += a p_{i-1}, and partial sums of (p_i, q_i), (r_i, q_i), then (q_i, q_i),
// (r_i, r_i) for one reduction: pair h, sum j at red[h grid 32 + blk 32 +
// j 16 + k].
template <int RC>
__device__ void f_dots2(const Ctx &c, const double (&acc)[2][RC], int pair) {
  __shared__ double sred[CG_WARPS][2][16];
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int k = 0; k < RC; ++k) sred[threadIdx.x >> 5][j][k] = acc[j][k];
  __syncthreads();
  if (threadIdx.x < 2 * RC) {
    const int j = threadIdx.x / RC, k = threadIdx.x % RC;
    double sm = 0.0;
    for (int w = 0; w < CG_WARPS; ++w) sm += sred[w][j][k];
    c.red[(long long)pair * gridDim.x * 32 + (long long)blockIdx.x * 32 + j * 16 + k] = sm;
  }
  __syncthreads();
}

template <int RC>
__device__ void f_step_dots(const Ctx &c, float *Rv, float *Pv, float *Dv, const float *Qo, const float *Qn,
                            const float *a, const float *b) {
  const int R = c.R;
  double acc[2][RC];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[j][k] = 0.0;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
    const int col = e % R;
    const float pold = Pv[e];
    const float r = fmaf(-a[col], __ldcg(Qo + e), Rv[e]);
    const float pn = fmaf(b[col], pold, r);
    Dv[e] = fmaf(a[col], pold, Dv[e]);
    Rv[e] = r;
    Pv[e] = pn;
    const double q = (double)__ldcg(Qn + e);
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k == col) {
        acc[0][k] += (double)pn * q;
        acc[1][k] += (double)r * q;
      }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) warp_sum<RC>(acc[j]);
  f_dots2<RC>(c, acc, 0);
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[j][k] = 0.0;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {  // this thread's own r_i, just stored
    const int col = e % R;
    const double q = (double)__ldcg(Qn + e), r = (double)Rv[e];
#pragma unroll
    for (int k = 0; k < RC; ++k)
      if (k == col) {
        acc[0][k] += q * q;
        acc[1][k] += r * r;
      }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) warp_sum<RC>(acc[j]);
  f_dots2<RC>(c, acc, 1);
}

// FP32 CG on S32 d = r (r already in F_R, d accumulates in F_D from 0), per
// column until |r_k| <= tol_in |r_k(0)|; returns iterations or -1 (timeout).
// One grid-wide reduction per iteration (the application's own barriers
// aside): after q_i = S32 p_i the owners update r, p, d and reduce
// (p_i, q_i), (r_i, q_i), (q_i, q_i), (r_i, r_i) together; alpha_i =
// (r_i, r_i) / (p_i, q_i), and |r_{i+1}|^2 = (r_i, r_i) - 2 alpha_i (r_i, q_i) +
// alpha_i^2 (q_i, q_i) gives beta_i and the stopping test before r_{i+1} is
// formed (by the next iteration's owners, from the vectors of this one).
template <int RC>
__device__ int f_cg(const Ctx &c, const double *tol_in, int max_it) {
  __shared__ double s_r0[16], s_rn[16], s_d[4][16];
  __shared__ float s_a[16], s_b[16];
  __shared__ int s_done;
  float *Rv = c.fdl[F_R], *Dv = c.fdl[F_D], *Pv = c.fdl[F_P0];
  float *Qb[2] = {c.fdl[F_Q], c.fdl[F_P1]};
  const int R = c.R;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
    Pv[e] = 0.f;
    Qb[0][e] = 0.f;
    Dv[e] = 0.f;
  }
  f_partial_dot<RC>(c, Rv, Rv, 1);
  if (!grid_sync(c)) return -1;
  finish_dot<RC>(c, 1, s_rn);
  if (threadIdx.x < 16) {
    s_r0[threadIdx.x] = threadIdx.x < RC ? s_rn[threadIdx.x] : 0.0;
    s_a[threadIdx.x] = 0.f;  // p_0 = r_0: no previous direction
    s_b[threadIdx.x] = 0.f;
  }
  __syncthreads();
  int it = 0, cur = 0;
  while (true) {
    if (threadIdx.x == 0) {
      int done = 1;
      for (int k = 0; k < R && k < RC; ++k)
        if (s_r0[k] > 0.0 && s_rn[k] > tol_in[k] * tol_in[k] * s_r0[k]) done = 0;
      s_done = done || it >= max_it;
    }
    __syncthreads();
    if (s_done) break;
    const DirIn dir{Rv, Qb[cur], Pv, s_a, s_b};
    if (!f_apply_S<RC>(c, dir, Qb[cur ^ 1])) return -1;
    f_step_dots<RC>(c, Rv, Pv, Dv, Qb[cur], Qb[cur ^ 1], s_a, s_b);
    if (!grid_sync(c)) return -1;
    if (threadIdx.x < 4 * RC) {
      const int j = threadIdx.x / RC, k = threadIdx.x % RC;
      const long long base = (long long)(j >> 1) * gridDim.x * 32;
      double sm = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) sm += ldg_cg(c.red + base + (long long)b * 32 + (j & 1) * 16 + k);
      s_d[j][k] = sm;
    }
    __syncthreads();
    if (threadIdx.x < RC) {
      const int k = threadIdx.x;
      const double pq = s_d[0][k], rq = s_d[1][k], qq = s_d[2][k], rr = s_d[3][k];
      const bool live = k < R && s_r0[k] > 0.0 && rr > tol_in[k] * tol_in[k] * s_r0[k] && pq != 0.0;
      const double al = live ? rr / pq : 0.0;
      const double rn = live ? fmax(rr - 2.0 * al * rq + al * al * qq, 0.0) : rr;
      s_a[k] = (float)al;
      s_b[k] = (live && rr > 0.0) ? (float)(rn / rr) : 0.f;
      s_rn[k] = rn;
    }
    __syncthreads();
    cur ^= 1;
    ++it;
  }
  // the pending step d += alpha_i p_i of the last reduction
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) Dv[e] = fmaf(s_a[e % R], Pv[e], Dv[e]);
  return it;
}

// MIXED solve of S_theta mu = B: FP64 residuals, FP32 corrections.  Returns the
// inner iterations or -1; s_bn receives |B| per column.
template <int RC>
__device__ int refine_solve(const Ctx &c, double *s_bn) {
  __shared__ double s_rn[16];
  __shared__ int s_done;
  double *B = c.dl[V_B], *MU = c.dl[V_MU], *RES = c.dl[V_RES], *Q = c.dl[V_Q];
  const int R = c.R;
  for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
    MU[e] = 0.0;
    RES[e] = B[e];
  }
  partial_dot<RC>(c, B, B, 0);
  if (!grid_sync(c)) return -1;
  finish_dot<RC>(c, 0, s_bn);
  if (threadIdx.x < RC) {
    s_rn[threadIdx.x] = s_bn[threadIdx.x];
    s_bn[threadIdx.x] = sqrt(s_bn[threadIdx.x]);
  }
  __syncthreads();
  // each sweep reduces its residual by tol_in: 1e-5 (about what the FP32
  // operator allows), or only as far as the target needs (with a margin of 3)
  __shared__ double s_tin[16];
  int total = 0, sweeps = 0;
  while (true) {
    if (threadIdx.x == 0) {
      int done = 1;
      for (int k = 0; k < R && k < RC; ++k)
        if (s_bn[k] > 0.0 && sqrt(s_rn[k]) >= c.tol * s_bn[k]) done = 0;
      s_done = done || sweeps >= c.max_refine || total >= c.max_iters;
    }
    __syncthreads();
    if (s_done) break;
    if (threadIdx.x < RC) {
      const int k = threadIdx.x;
      const double rn = sqrt(s_rn[k]);
      s_tin[k] = rn > 0.0 ? fmax(1e-5, fmin(0.5, 0.3 * c.tol * s_bn[k] / rn)) : 1e-5;
    }
    __syncthreads();
    // r32 = RES / |RES| per column (columns already converged: 0)
    for (int e = gthread(); e < c.n_dl * R; e += nthreads()) {
      const int k = e % R;
      const double rn = sqrt(s_rn[k]);
      const bool live = s_bn[k] > 0.0 && rn >= c.tol * s_bn[k];
      c.fdl[F_R][e] = live ? (float)(RES[e] / rn) : 0.f;
    }
    if (!grid_sync(c)) return -1;
    const int it = f_cg<RC>(c, s_tin, c.max_iters - total);
    if (it < 0) return -1;
    total += it;
    ++sweeps;
    for (int e = gthread(); e < c.n_dl * R; e += nthreads())
      MU[e] = fma(sqrt(s_rn[e % R]), (double)c.fdl[F_D][e], MU[e]);
    if (!grid_sync(c)) return -1;
    if (!apply_S<RC>(c, MU, Q)) return -1;
    for (int e = gthread(); e < c.n_dl * R; e += nthreads()) RES[e] = B[e] - ldg_cg(Q + e);
    partial_dot<RC>(c, RES, RES, 0);
    if (!grid_sync(c)) return -1;
    finish_dot<RC>(c, 0, s_rn);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c.info[33] = sweeps;
  return total;
}

template <int RC>
__device__ void forward_program(const Ctx &c) {
  __shared__ double s_bn[16], s_rn[16];
  double *B = c.dl[V_B], *MU = c.dl[V_MU], *Q = c.dl[V_Q];
  if (c.mode == 3) {  // S_theta mu = B for a given B (tangent and other interface solves)
    const int it = c.fb ? refine_solve<RC>(c, s_bn) : cg_solve<RC>(c, s_bn);
    if (it < 0) return;
    if (!apply_S<RC>(c, MU, Q)) return;
    for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) c.dl[V_TMP][e] = B[e] - ldg_cg(Q + e);
    partial_dot<RC>(c, c.dl[V_TMP], c.dl[V_TMP], 0);
    if (!grid_sync(c)) return;
    finish_dot<RC>(c, 0, s_rn);
    if (blockIdx.x == 0 && threadIdx.x < RC && threadIdx.x < c.R)
      c.info[1 + threadIdx.x] = s_bn[threadIdx.x] > 0.0 ? sqrt(s_rn[threadIdx.x]) / s_bn[threadIdx.x] : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) c.info[0] = it;
    return;
  }
  // ---------------- right-hand side b_theta
  // dpi = -sum a_Pi ; ppi = sum p_Pi (a, p are the per-subdomain A_m y and Q_Gamma Q^T f)
  for (int e = gthread(); e < c.n_pi * c.R; e += nthreads()) {
    const int p = e / c.R, k = e % c.R;
    double ad = 0.0, pp = 0.0;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      ad += c.db[d.oAy + (long long)a * c.R + k];
      pp += c.db[d.oP + (long long)a * c.R + k];
    }
    c.pv[P_DPI][e] = -ad;
    c.pv[P_PPI][e] = pp;
  }
  if (!grid_sync(c)) return;
  // mpf = S_Pi^{-1}(ppi + D^T dpi) ; gf = dpi - D mpf
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_PPI], c.o_C1, c.pv[P_DPI], 1.0, c.pv[P_MPF], c.o_C2, c.pv[P_DPI], c.o_C3,
              c.pv[P_PPI], -1.0, c.pv[P_GF]);
  if (!grid_sync(c)) return;
  ph_dl_first<RC>(c, c.pv[P_MPF], nullptr, c.pv[P_GF], 1);
  if (!grid_sync(c)) return;
  if (!second_half<RC>(c, B)) return;
  int it = 0;
  if (c.mode == 2) {  // mu given: only |b| for the relative residual
    partial_dot<RC>(c, B, B, 0);
    if (!grid_sync(c)) return;
    finish_dot<RC>(c, 0, s_bn);
    if (threadIdx.x < RC) s_bn[threadIdx.x] = sqrt(s_bn[threadIdx.x]);
    __syncthreads();
  } else {
    it = c.fb ? refine_solve<RC>(c, s_bn) : cg_solve<RC>(c, s_bn);
    if (it < 0) return;
  }
  // ---------------- true residual |b - S mu| / |b|
  if (!apply_S<RC>(c, MU, Q)) return;
  for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) c.dl[V_TMP][e] = B[e] - ldg_cg(Q + e);
  partial_dot<RC>(c, c.dl[V_TMP], c.dl[V_TMP], 0);
  if (!grid_sync(c)) return;
  finish_dot<RC>(c, 0, s_rn);
  if (blockIdx.x == 0 && threadIdx.x < RC && threadIdx.x < c.R) {
    c.info[1 + threadIdx.x] = s_bn[threadIdx.x] > 0.0 ? sqrt(s_rn[threadIdx.x]) / s_bn[threadIdx.x] : 0.0;
    c.info[17 + threadIdx.x] = s_bn[threadIdx.x];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c.info[0] = it;
  // ---------------- reconstruction, Eq. (coarse_sol_2)
  ph_pi_rows<RC>(c, MU);
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_H1, 1.0, c.pv[P_PSI2], S_H2, 1.0, c.pv[P_S2]);
  if (!grid_sync(c)) return;
  // mu_Pi = mpf + S_Pi^{-1} s2 - C1 psi2
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_S2], c.o_C1, c.pv[P_PSI2], -1.0, c.pv[P_MPIF], -1, nullptr, -1, nullptr,
              0.0, nullptr);
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < c.n_pi * c.R; e += nthreads()) {
    const double v = c.pv[P_MPIF][e] + c.pv[P_MPF][e];
    c.pv[P_MPIF][e] = v;
    if (c.mu_out) c.mu_out[e] = v;
  }
  if (c.mu_out)
    for (int e = gthread(); e < c.n_dl * c.R; e += nthreads()) c.mu_out[(long long)c.n_pi * c.R + e] = MU[e];
  if (!grid_sync(c)) return;
  // c = y + K^+ E_Gamma [mu_Pi^; mu_Delta^]
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tc; t += nwarps()) {
    const int s = c.ints[c.o_tc + 2 * t], j = c.ints[c.o_tc + 2 * t + 1];
    const SubDev d = c.subs[s];
    const double *row = c.db + d.oKpE + (long long)j * d.nG;
    const int *gpi = c.ints + d.gpi_off;
    const int *gdl = c.ints + d.gdl_off;
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int b = lane; b < d.nG; b += 32) {
      const double m = row[b];
      const double *src = b < d.nPi ? c.pv[P_MPIF] + (long long)gpi[b] * c.R : MU + (long long)gdl[b - d.nPi] * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(m, ldg_cg(src + k), acc[k]);
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) {
          const double v = c.db[d.oY + (long long)j * c.R + k] + acc[k];
          c.db[d.oC + (long long)j * c.R + k] = v;
          if (c.c_out) c.c_out[(d.w_off + j) * c.R + k] = v;
        }
    }
  }
}

// Adjoint of the solve map (f, g) -> c for a cotangent c-bar held in the
// per-subdomain C buffers (and copied into the y buffers): every step of the
// forward program transposed in reverse order; S_theta, S_Pi^{-1} and
// C2 = I - D S_Pi^{-1} D^T are symmetric, C1^T = C3.  Leaves a-bar in the
// A_m y buffers and p-bar in the p buffers for the local products that follow.
template <int RC>
__device__ void adjoint_program(const Ctx &c) {
  __shared__ double s_bn[16];
  double *B = c.dl[V_B], *MU = c.dl[V_MU];
  const int lane = threadIdx.x & 31;
  // lambda-bar = (K^+ E)^T c-bar on every Gamma row
  for (int t = gwarp(); t < c.n_tg; t += nwarps()) {
    const int s = c.ints[c.o_tg + 2 * t], a = c.ints[c.o_tg + 2 * t + 1];
    const SubDev d = c.subs[s];
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int j = lane; j < d.M; j += 32) {
      const double m = c.db[d.oKpE + (long long)j * d.nG + a];
      const double *src = c.db + d.oC + (long long)j * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(m, src[k], acc[k]);
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
      double *o = slab_row(c, S_H1, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) o[k] = acc[k];
    }
  }
  if (!grid_sync(c)) return;
  // mu-bar_Pi (gathered), mu-bar_Delta direct part
  ph_pi_gather(c, S_H1, 1.0, c.pv[P_MPIF], -1, 0.0, nullptr);
  ph_dl_gather(c, S_H1, 1.0, c.dl[V_TMP], nullptr, 0.0, -1, nullptr);
  if (!grid_sync(c)) return;
  // s2-bar = S_Pi^{-1} mu-bar_Pi ; (C3 mu-bar_Pi) for psi2-bar = -C3 mu-bar_Pi
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_MPIF], -1, nullptr, 0.0, c.pv[P_S2], c.o_C3, c.pv[P_MPIF], -1, nullptr, 0.0,
              c.pv[P_PSI2]);
  if (!grid_sync(c)) return;
  // mu-bar = direct + sum R_D^T (Psi_DPi s2-bar^ - Lambda_PiD^T (C3 mu-bar_Pi)^)
  ph_dl_last<RC>(c, c.pv[P_S2], c.pv[P_PSI2], false);
  if (!grid_sync(c)) return;
  ph_dl_gather(c, S_YL, 1.0, B, c.dl[V_TMP], 1.0, -1, nullptr);
  if (!grid_sync(c)) return;
  // b-bar = S_theta^{-1} mu-bar
  const int it = cg_solve<RC>(c, s_bn);
  if (it < 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) c.info[0] = it;
  // dt-bar = W D~ b-bar (first half of the operator applied to b-bar)
  ph_pi_rows<RC>(c, MU);
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_H1, 1.0, c.pv[P_PSI], S_H2, -1.0, c.pv[P_RA]);
  if (!grid_sync(c)) return;
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_RA], c.o_C1, c.pv[P_PSI], 1.0, c.pv[P_MPI], c.o_C2, c.pv[P_PSI], c.o_C3,
              c.pv[P_RA], -1.0, c.pv[P_G]);
  if (!grid_sync(c)) return;
  ph_dl_first<RC>(c, c.pv[P_MPI], MU, c.pv[P_G], 0);
  if (!grid_sync(c)) return;
  if (!apply_W<RC>(c)) return;  // V_W = dt-bar
  // H1 = Lambda_PiD b-bar^ , H2 = Psi_PiD b-bar^ , ZL = Lambda^T [0; dt-bar^]
  ph_pi_rows<RC>(c, MU);
  ph_g_lamT<RC>(c, c.dl[V_W]);
  if (!grid_sync(c)) return;
  // gf-bar = sum H1 ; mpf-bar = mu-bar_Pi + sum H2 - sum ZL_Pi
  for (int e = gthread(); e < c.n_pi * c.R; e += nthreads()) {
    const int p = e / c.R, k = e % c.R;
    double g1 = 0.0, h2 = 0.0, z = 0.0;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      g1 += ldg_cg(slab_row(c, S_H1, d, a) + k);
      h2 += ldg_cg(slab_row(c, S_H2, d, a) + k);
      z += ldg_cg(slab_row(c, S_ZL, d, a) + k);
    }
    c.pv[P_GF][e] = g1;
    c.pv[P_MPF][e] = ldg_cg(c.pv[P_MPIF] + e) + h2 - z;
  }
  if (!grid_sync(c)) return;
  // ppi-bar = S_Pi^{-1} mpf-bar - C1 gf-bar ; dpi-bar = C3 mpf-bar + C2 gf-bar
  if (c.n_pi > 0)
    ph_coarse(c, c.o_Sinv, c.pv[P_MPF], c.o_C1, c.pv[P_GF], -1.0, c.pv[P_PPI], c.o_C3, c.pv[P_MPF], c.o_C2,
              c.pv[P_GF], 1.0, c.pv[P_DPI]);
  if (!grid_sync(c)) return;
  // a-bar = [-R_Pi dpi-bar ; -R_D dt-bar], p-bar = [R_Pi ppi-bar ; R_D b-bar]
  for (int e = gthread(); e < c.n_tg * c.R; e += nthreads()) {
    const int t = e / c.R, k = e % c.R;
    const int s = c.ints[c.o_tg + 2 * t], a = c.ints[c.o_tg + 2 * t + 1];
    const SubDev &d = c.subs[s];
    double ab, pb;
    if (a < d.nPi) {
      const int gp = c.ints[d.gpi_off + a];
      ab = -ldg_cg(c.pv[P_DPI] + (long long)gp * c.R + k);
      pb = ldg_cg(c.pv[P_PPI] + (long long)gp * c.R + k);
    } else {
      const int gd = c.ints[d.gdl_off + a - d.nPi];
      ab = -ldg_cg(c.dl[V_W] + (long long)gd * c.R + k);
      pb = ldg_cg(MU + (long long)gd * c.R + k);
    }
    c.db[d.oAy + (long long)a * c.R + k] = ab;
    c.db[d.oP + (long long)a * c.R + k] = pb;
  }
  (void)B;
}

// Pi rows of (K^+ E_Gamma)^T c-hat into slab H1 (c-hat in the coefficient buffers)
template <int RC>
__device__ void ph_pi_kpe(const Ctx &c) {
  const int lane = threadIdx.x & 31;
  for (int t = gwarp(); t < c.n_tpi; t += nwarps()) {
    const int s = c.ints[c.o_tpi + 2 * t], a = c.ints[c.o_tpi + 2 * t + 1];
    const SubDev d = c.subs[s];
    double acc[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) acc[k] = 0.0;
    for (int j = lane; j < d.M; j += 32) {
      const double m = c.db[d.oKpE + (long long)j * d.nG + a];
      const double *src = c.db + d.oC + (long long)j * c.R;
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) acc[k] = fma(m, src[k], acc[k]);
    }
    warp_sum<RC>(acc);
    if (lane == 0) {
      double *o = slab_row(c, S_H1, d, a);
#pragma unroll
      for (int k = 0; k < RC; ++k)
        if (k < c.R) o[k] = acc[k];
    }
  }
}

// Interface vectors of the scale gradient (run after the adjoint solve; mu in
// V_MU, b-bar = S_theta^{-1} mu-bar in the bank, c-hat and the forward y, p,
// a = A_m y in the subdomain buffers).  The derivative of
//   c-hat^T c(mu, s) + b-bar^T (b_theta(s) - S_theta(s) mu)
// at fixed mu (= dL/ds, since S_theta b-bar = mu-bar) is a sum over every
// application of a local operator in the right-hand side, in S_theta mu and in
// the reconstruction of (cotangent of its output) x (its input)^T.  The reverse
// passes of the right-hand side and of S_theta mu share their second half up
// to sign (cotangents b-bar and -b-bar), so one pass with b-bar serves both;
// the pairs then merge into four Lambda, two Psi and two Phi pairs per
// right-hand side, stored here as interface vectors (see scale_plan.cpp), and
// the cotangents of the four coarse matrices S_Pi^{-1}, C1, C2, C3 are formed
// in full.
template <int RC>
__device__ void scale_program(const Ctx &c) {
  const int R = c.R, nPR = c.n_pi * R, nDR = c.n_dl * R;
  const long long nd = c.n_dl > 0 ? c.n_dl : 1, np = c.n_pi > 0 ? c.n_pi : 1;
  auto BD = [&](int k) { return c.bkd + (long long)k * nd * R; };
  auto BP = [&](int k) { return c.bkp + (long long)k * np * R; };
  double *MU = c.dl[V_MU], *B = c.dl[V_B], *Q = c.dl[V_Q];
  const bool coarse = c.n_pi > 0;
  // ---- the right-hand side program (forward)
  for (int e = gthread(); e < nPR; e += nthreads()) {
    const int p = e / R, k = e % R;
    double ad = 0.0, pp = 0.0;
    for (int o = 0; o < 4; ++o) {
      const int s = c.ints[c.o_pi_own + 8 * p + 2 * o];
      if (s < 0) continue;
      const int a = c.ints[c.o_pi_own + 8 * p + 2 * o + 1];
      const SubDev &d = c.subs[s];
      ad += c.db[d.oAy + (long long)a * R + k];
      pp += c.db[d.oP + (long long)a * R + k];
    }
    c.pv[P_DPI][e] = -ad;
    c.pv[P_PPI][e] = pp;
  }
  if (!grid_sync(c)) return;
  if (coarse)
    ph_coarse(c, c.o_Sinv, c.pv[P_PPI], c.o_C1, c.pv[P_DPI], 1.0, c.pv[P_MPF], c.o_C2, c.pv[P_DPI], c.o_C3,
              c.pv[P_PPI], -1.0, c.pv[P_GF]);
  if (!grid_sync(c)) return;
  ph_dl_first<RC>(c, c.pv[P_MPF], nullptr, c.pv[P_GF], 1);
  if (!grid_sync(c)) return;
  if (!second_half<RC>(c, B)) return;
  for (int e = gthread(); e < nDR; e += nthreads()) {
    BD(SD_VR)[e] = c.dl[V_V][e];
    BD(SD_PVR)[e] = c.dl[V_PV][e];
    BD(SD_WR)[e] = c.dl[V_W][e];
    BD(SD_MU)[e] = MU[e];
    BD(SD_NEGBB)[e] = -BD(SD_BB)[e];
  }
  for (int e = gthread(); e < nPR; e += nthreads()) {
    BP(SP_DPI)[e] = c.pv[P_DPI][e];
    BP(SP_PPI)[e] = c.pv[P_PPI][e];
    BP(SP_MPF)[e] = c.pv[P_MPF][e];
    BP(SP_GF)[e] = c.pv[P_GF][e];
    BP(SP_RNUR)[e] = c.pv[P_RNU][e];
    BP(SP_NUR)[e] = c.pv[P_NU][e];
    BP(SP_DNUR)[e] = c.pv[P_DNU][e];
    BP(SP_ZERO)[e] = 0.0;
  }
  if (!grid_sync(c)) return;
  // ---- S_theta mu (forward), and its combinations with the right-hand side's vectors
  if (!apply_S<RC>(c, MU, Q)) return;
  for (int e = gthread(); e < nDR; e += nthreads()) {
    BD(SD_WRS)[e] = BD(SD_WR)[e] - c.dl[V_W][e];
    BD(SD_PVSR)[e] = c.dl[V_PV][e] - BD(SD_PVR)[e];
    BD(SD_VSR)[e] = c.dl[V_V][e] - BD(SD_VR)[e];
  }
  for (int e = gthread(); e < nPR; e += nthreads()) {
    const double mpf = BP(SP_MPF)[e];
    BP(SP_PIA)[e] = c.pv[P_DNU][e] - c.pv[P_G][e] - BP(SP_DNUR)[e] + BP(SP_GF)[e];
    BP(SP_PIC)[e] = c.pv[P_MPI][e] - mpf;
    BP(SP_PID)[e] = BP(SP_NUR)[e] - c.pv[P_NU][e] + mpf - c.pv[P_MPI][e];
    BP(SP_RNURS)[e] = BP(SP_RNUR)[e] - c.pv[P_RNU][e];
    BP(SP_RAS)[e] = c.pv[P_RA][e];
    BP(SP_PSIS)[e] = c.pv[P_PSI][e];
    BP(SP_DPIPSI)[e] = BP(SP_DPI)[e] - c.pv[P_PSI][e];
    BP(SP_RAPPI)[e] = c.pv[P_RA][e] - BP(SP_PPI)[e];
  }
  if (!grid_sync(c)) return;
  // ---- reconstruction (forward): psi2, s2, mu_Pi = mpf + S_Pi^{-1} s2 - C1 psi2
  ph_pi_rows<RC>(c, MU);
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_H1, 1.0, BP(SP_PSI2), S_H2, 1.0, BP(SP_S2));
  if (!grid_sync(c)) return;
  if (coarse)
    ph_coarse(c, c.o_Sinv, BP(SP_S2), c.o_C1, BP(SP_PSI2), -1.0, BP(SP_MPIF), -1, nullptr, -1, nullptr, 0.0,
              nullptr);
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < nPR; e += nthreads()) BP(SP_MPIF)[e] += BP(SP_MPF)[e];
  // ---- reverse of the reconstruction: mpif-bar = (K^+ E)^T c-hat on Pi, s2-bar, psi2-bar
  ph_pi_kpe<RC>(c);
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_H1, 1.0, BP(SP_MPIFB), -1, 0.0, nullptr);
  if (!grid_sync(c)) return;
  if (coarse)
    ph_coarse(c, c.o_Sinv, BP(SP_MPIFB), -1, nullptr, 0.0, BP(SP_S2B), c.o_C3, BP(SP_MPIFB), -1, nullptr, 0.0,
              BP(SP_PSI2B));
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < nPR; e += nthreads()) BP(SP_PSI2B)[e] = -BP(SP_PSI2B)[e];
  // ---- the second half reversed with b-bar: nu-bar, dnu-bar, rnu-bar, w-bar, pv-bar, v-bar
  ph_pi_rows<RC>(c, BD(SD_BB));
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_H1, 1.0, BP(SP_GFB), S_H2, 1.0, BP(SP_NUB));
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < nPR; e += nthreads()) BP(SP_DNUB)[e] = -BP(SP_GFB)[e];
  if (!grid_sync(c)) return;
  if (coarse)
    ph_coarse(c, c.o_Sinv, BP(SP_NUB), c.o_C1, BP(SP_DNUB), 1.0, BP(SP_RNUB), -1, nullptr, -1, nullptr, 0.0,
              nullptr);
  if (!grid_sync(c)) return;
  ph_dl_first<RC>(c, BP(SP_RNUB), BD(SD_NEGBB), BP(SP_ZERO), 0);  // VL = -(Lambda L(rnu-bar, b-bar))_Delta
  if (!grid_sync(c)) return;
  ph_dl_gather(c, S_VL, -1.0, BD(SD_WB), nullptr, 0.0, -1, nullptr);
  if (!grid_sync(c)) return;
  ph_dl_phi<RC>(c, false, BD(SD_WB), S_TL);  // -Phi w-bar^
  if (!grid_sync(c)) return;
  ph_dl_gather(c, S_TL, c.theta, BD(SD_PVB), nullptr, 0.0, -1, nullptr);
  if (!grid_sync(c)) return;
  ph_dl_phi<RC>(c, true, BD(SD_PVB), S_T2L);  // -Phi^T pv-bar^
  if (!grid_sync(c)) return;
  ph_dl_gather(c, S_T2L, 1.0, BD(SD_VB), BD(SD_WB), 1.0 - c.theta, -1, nullptr);
  if (!grid_sync(c)) return;
  // ---- the first halves reversed: mpf-bar (right-hand side), mpi-bar (S_theta mu)
  ph_g_lamT<RC>(c, BD(SD_VB));
  if (!grid_sync(c)) return;
  ph_pi_gather(c, S_ZL, 1.0, BP(SP_ZLV), -1, 0.0, nullptr);
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < nPR; e += nthreads()) {
    const double zl = BP(SP_ZLV)[e], nu = BP(SP_NUB)[e];
    BP(SP_MPFB)[e] = BP(SP_MPIFB)[e] - zl + nu;
    BP(SP_MPIBS)[e] = zl - nu;
  }
  if (!grid_sync(c)) return;
  if (coarse) {
    ph_coarse(c, c.o_Sinv, BP(SP_MPIBS), c.o_C1, BP(SP_DNUB), -1.0, BP(SP_RABS), c.o_C3, BP(SP_MPIBS), c.o_C2,
              BP(SP_DNUB), 1.0, BP(SP_PSIBS));
    if (!grid_sync(c)) return;
    ph_coarse(c, c.o_Sinv, BP(SP_MPFB), c.o_C1, BP(SP_GFB), -1.0, BP(SP_PPIB), c.o_C3, BP(SP_MPFB), c.o_C2,
              BP(SP_GFB), 1.0, BP(SP_DPIB));
  }
  if (!grid_sync(c)) return;
  for (int e = gthread(); e < nPR; e += nthreads()) {
    BP(SP_PIB)[e] = BP(SP_PSIBS)[e] + BP(SP_PSI2B)[e];
    BP(SP_PIE)[e] = BP(SP_S2B)[e] - BP(SP_RABS)[e];
  }
  // ---- cotangents of the coarse matrices (sums of outer products over the columns)
  const int n = c.n_pi;
  for (long long e = gthread(); e < (long long)n * n; e += nthreads()) {
    const int p = int(e / n), q = int(e % n);
    double sb = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    for (int k = 0; k < R; ++k) {
      const long long ip = (long long)p * R + k, iq = (long long)q * R + k;
      sb += BP(SP_NUB)[ip] * BP(SP_RNURS)[iq] + BP(SP_MPIBS)[ip] * BP(SP_RAS)[iq] +
            BP(SP_MPFB)[ip] * BP(SP_PPI)[iq] + BP(SP_MPIFB)[ip] * BP(SP_S2)[iq];
      c1 += BP(SP_MPIBS)[ip] * BP(SP_PSIS)[iq] + BP(SP_MPFB)[ip] * BP(SP_DPI)[iq] -
            BP(SP_MPIFB)[ip] * BP(SP_PSI2)[iq];
      c2 += BP(SP_GFB)[ip] * BP(SP_DPIPSI)[iq];
      c3 += BP(SP_GFB)[ip] * (BP(SP_RAPPI)[iq] - BP(SP_RNURS)[iq]);
    }
    c.csb[e] = sb;
    c.cc1b[e] = c1;
    c.cc2b[e] = c2;
    c.cc3b[e] = c3;
  }
}

template <int RC>
__global__ void __launch_bounds__(CG_THREADS, 1) cg_kernel(Ctx c) {
  if (c.mode == 1)
    adjoint_program<RC>(c);
  else if (c.mode == 4)
    scale_program<RC>(c);
  else
    forward_program<RC>(c);  // 0 solve, 2 residual at a given mu, 3 solve for a given right-hand side
}

}  // namespace

// the CG region's mu, right-hand side and residual Delta vectors ([n_dl x R] each)
void cg_vectors(const Plan &p, void *ws, double **mu, double **rhs, double **res) {
  double *db = reinterpret_cast<double *>(static_cast<char *>(ws) + p.off_dbl);
  const long long nd = p.n_dl > 0 ? p.n_dl : 1, R = p.n_rhs;
  double *cg = db + p.o_cg;
  *mu = cg + V_MU * nd * R;
  *rhs = cg + V_B * nd * R;
  *res = cg + V_TMP * nd * R;
}

cudaError_t launch_cg(const Plan &p, void *ws, const CgArgs &a, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  Ctx c;
  c.subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  c.ints = reinterpret_cast<const int *>(base + p.off_ints);
  c.db = reinterpret_cast<double *>(base + p.off_dbl);
  c.n_sub = p.n_sub;
  c.n_pi = p.n_pi;
  c.n_dl = p.n_dl;
  c.R = p.n_rhs;
  c.o_pi_own = p.o_pi_own;
  c.o_dl_own = p.o_dl_own;
  c.o_tpi = p.o_tasks_pi;
  c.n_tpi = p.n_tasks_pi;
  c.o_tdl = p.o_tasks_dl;
  c.n_tdl = p.n_tasks_dl;
  c.o_tg = p.o_tasks_g;
  c.n_tg = p.n_tasks_g;
  c.o_tc = p.o_tasks_c;
  c.n_tc = p.n_tasks_c;
  c.o_dl_rows = p.o_dl_rows;
  c.o_gam_rows = p.o_gam_rows;
  c.o_Sinv = p.o_Sinv;
  c.o_C1 = p.o_C1;
  c.o_C2 = p.o_C2;
  c.o_C3 = p.o_C3;
  const long long nd = p.n_dl > 0 ? p.n_dl : 1, np = p.n_pi > 0 ? p.n_pi : 1, R = p.n_rhs;
  double *cg = c.db + p.o_cg;
  for (int k = 0; k < N_DLVEC; ++k) c.dl[k] = cg + k * nd * R;
  cg += N_DLVEC * nd * R;
  for (int k = 0; k < N_PIVEC; ++k) c.pv[k] = cg + k * np * R;
  cg += N_PIVEC * np * R;
  c.red = cg;              // 2048 x 32 doubles reserved below
  c.info = cg + 2048 * 32 - 64;
  for (int k = 0; k < N_SLAB; ++k) c.slab[k] = c.db + p.o_loc + (long long)k * p.sum_nG * R;
  c.bar = reinterpret_cast<unsigned *>(c.db + p.o_status + 2 * p.n_sub + 8);
  c.err = reinterpret_cast<int *>(c.db + p.o_status + 2 * p.n_sub + 16);
  c.theta = a.theta;
  c.tol = a.tol;
  c.max_iters = a.max_iters;
  c.mu_out = a.mu_out;
  c.c_out = a.c_out;
  c.mode = a.mode;
  c.max_refine = a.max_refine;
  c.bar_limit_ns = p.opt.barrier_timeout_ms > 0 ? 1000000ull * (unsigned long long)p.opt.barrier_timeout_ms
                                                : 2000000000ull;
  c.bar_extra = p.opt.inject_barrier_stall ? 1u : 0u;
  c.bkd = c.db + p.o_bank_dl;
  c.bkp = c.db + p.o_bank_pi;
  c.csb = c.db + p.o_cSb;
  c.cc1b = c.db + p.o_cC1b;
  c.cc2b = c.db + p.o_cC2b;
  c.cc3b = c.db + p.o_cC3b;
  c.fb = nullptr;
  if (p.mixed && p.o_f32 >= 0 && (a.mode == 0 || a.mode == 3)) {
    c.fb = reinterpret_cast<float *>(c.db + p.o_f32);
    c.f_Sinv = p.f_Sinv;
    c.f_C1 = p.f_C1;
    c.f_C2 = p.f_C2;
    c.f_C3 = p.f_C3;
    for (int k = 0; k < N_FDL; ++k) c.fdl[k] = c.fb + p.f_dl + k * nd * R;
    for (int k = 0; k < N_FPV; ++k) c.fpv[k] = c.fb + p.f_pv + k * np * R;
    for (int k = 0; k < N_FSLAB; ++k) c.fslab[k] = c.fb + p.f_slab + (long long)k * p.sum_nG * R;
  }
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // at most 1022 CTAs: the inner CG's four per-CTA partial sums use twice
  // the 32 entries per CTA of the 2048 x 32 reduction area (its last 64: info)
  const int grid = nsm < 1022 ? nsm : 1022;
  void *args[] = {&c};
  DDELM_COUNT_LAUNCH();
  if (p.n_rhs == 1) return cudaLaunchCooperativeKernel((const void *)cg_kernel<1>, grid, CG_THREADS, args, 0, s);
  return cudaLaunchCooperativeKernel((const void *)cg_kernel<16>, grid, CG_THREADS, args, 0, s);
}

}  // namespace ddelm
