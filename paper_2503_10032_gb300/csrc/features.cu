// Fused feature assembly (Sec. 2.2 and Sec. 2.2.1, Sec. 3.1, Sec. 3.2):
// phi_j(x) = tanh(w_j . x + b_j) and the rows of K_c^i, K-bar^i, A_m^i,
// A-bar^i and the evaluation matrix, written once in FP64 with coalesced
// row-major stores (consecutive threads -> consecutive neurons j).
//
//   L phi (Poisson)   = 2 |w|^2 t (1 - t^2)
//   L phi (diffusion) = 2 a |w|^2 t (1 - t^2) - (grad a . w)(1 - t^2)
//   B phi = C phi = t,   F phi = (w . n)(1 - t^2)
// with t = tanh(w . x + b) (tanh_half below).  The interior rows and the first pass over the
// other rows take one tanh per (point, neuron); the rows that combine point
// values or fluxes (change of variables, A_m corner rows) are formed from them.
#include <algorithm>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

// tanh(u / 2) in about 18 FP64 operations (the FP64 pipe of this GPU is the
// scarce unit of the feature kernels), absolute error below 2e-16:
//   E = exp(-|u|) by the table-driven method of Tang (ACM TOMS 15(2), 1989):
//   |u| = k ln2/256 + r with ln2/256 split as in Cody and Waite (hi with 39
//   significant bits, so that k hi is exact for k < 2^14), 2^(-j/256) from a
//   256-entry table (j = k mod 256) and exp(-r) from its degree-4 Taylor
//   polynomial (|r| <= ln2/512: remainder below 4e-17);
//   tanh(|u| / 2) = (1 - E) / (1 + E), the quotient from one Newton step on
//   an FP32 reciprocal of 1 + E in [1, 2] and one residual correction.
// |u| is clamped at 40 (tanh(20) rounds to 1); NaN propagates.
__device__ __forceinline__ double tanh_half(double u, const double *__restrict__ exp2tab) {
  const long long ub = __double_as_longlong(u);
  const long long ab = ub & 0x7FFFFFFFFFFFFFFFll;
  if (ab > 0x7FF0000000000000ll) return u;                      // NaN
  const double a = ab > 0x4044000000000000ll ? 40.0 : __longlong_as_double(ab);  // min(|u|, 40)
  const double inv_l = 0x1.71547652b82fep+8;      // 256 / ln 2
  const double l_hi = 0x1.62e42fefa4000p-9;       // ln 2 / 256, high part
  const double l_lo = -0x1.8432a1b0e2634p-51;     // ln 2 / 256 - l_hi
  const double shifter = 0x1.8p52;                // k lands in the low mantissa bits
  const double kt = fma(a, inv_l, shifter);
  const int k = __double2loint(kt);               // 0 <= k <= 14773
  const double kd = kt - shifter;
  double r = fma(-kd, l_hi, a);
  r = fma(-kd, l_lo, r);
  double q = fma(r, 1.0 / 24.0, -1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, -1.0);                            // exp(-r) = 1 + r q
  const double tj = exp2tab[k & 255];
  double e = fma(tj, r * q, tj);                  // 2^(-j/256) exp(-r)
  e = __hiloint2double(__double2hiint(e) - ((k >> 8) << 20), __double2loint(e));  // * 2^(-k/256 div)
  const double num = 1.0 - e, den = 1.0 + e;
  // FP32 reciprocal of den from its high word (20 mantissa bits), back to FP64
  const unsigned dh = (unsigned)__double2hiint(den);
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float((dh - 0x38000000u) << 3)));
  const unsigned yb = __float_as_uint(yf);
  double y = __hiloint2double((int)((yb >> 3) + 0x38000000u), (int)(yb << 29));
  y = fma(y, fma(-den, y, 1.0), y);               // relative error ~2^-40
  const double q0 = num * y;
  const double t = fma(fma(-den, q0, num), y, q0);
  return ub < 0 ? -t : t;
}

__device__ __forceinline__ void load_exp2tab(double *s, const double *__restrict__ g) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s[i] = g[i];
  __syncthreads();
}

// Interior collocation rows: rows [0, nI) of K_c^i and K-bar^i.
__global__ void __launch_bounds__(256) interior_rows_kernel(const SubDev *__restrict__ subs, int sub0,
                                                            double *__restrict__ db, long long o_w,
                                                            long long o_fc, long long o_exp2, long long o_xint,
                                                            long long o_aint, long long o_gaint, int op,
                                                            double w_int) {
  __shared__ double s_exp2[256];
  const SubDev d = subs[sub0 + blockIdx.y];
  const int r0 = blockIdx.x * 8;
  if (r0 >= d.nI) return;
  load_exp2tab(s_exp2, db + o_exp2);
  const double *w = db + o_w + 2 * d.w_off;
  const double4 *fc = reinterpret_cast<const double4 *>(db + o_fc) + d.w_off;
  for (int rr = 0; rr < 8; ++rr) {
    const int r = r0 + rr;
    if (r >= d.nI) break;
    const long long pi = d.int_off + r;
    const double x = db[o_xint + 2 * pi], y = db[o_xint + 2 * pi + 1];
    double a = 1.0, ax = 0.0, ay = 0.0;
    if (op == DDELM_OP_DIFFUSION) {
      a = db[o_aint + pi];
      ax = db[o_gaint + 2 * pi];
      ay = db[o_gaint + 2 * pi + 1];
    }
    double *o0 = db + d.oK + (long long)r * d.M;
    double *o1 = db + d.oKb + (long long)r * d.M;
    for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
      const double4 c = fc[j];  // 2 w_x, 2 w_y, 2 b, 2 |w|^2
      const double t = tanh_half(fma(c.x, x, fma(c.y, y, c.z)), s_exp2);
      const double s1 = fma(-t, t, 1.0);
      double v = (c.w * t) * s1;  // 2 |w|^2 t (1 - t^2)
      if (op == DDELM_OP_DIFFUSION) v = a * v - (ax * w[2 * j] + ay * w[2 * j + 1]) * s1;
      // Lap^2 phi = |w|^4 tanh''''(z) = 8 |w|^4 t (1 - t^2)(2 - 3 t^2), with c.w = 2 |w|^2,
      // weighted by w_int = H^4
      if (op == DDELM_OP_BIHARMONIC) v = w_int * (2.0 * (c.w * c.w) * (t * s1) * fma(-3.0 * t, t, 2.0));
      o0[j] = v;
      o1[j] = v;
    }
  }
}

// First pass over the special rows: one tanh per (point, neuron).
__global__ void __launch_bounds__(256) special_rows_kernel(const SpecialRow *__restrict__ rows,
                                                           const SubDev *__restrict__ subs,
                                                           double *__restrict__ db, long long o_w,
                                                           long long o_fc, long long o_exp2, double w_c1,
                                                           double w_f0, double w_f1) {
  __shared__ double s_exp2[256];
  const SpecialRow rw = rows[blockIdx.x];
  if (rw.kind == ROW_AM) return;
  load_exp2tab(s_exp2, db + o_exp2);
  const SubDev d = subs[rw.sub];
  const double *w = db + o_w + 2 * d.w_off;
  const double4 *fc = reinterpret_cast<const double4 *>(db + o_fc) + d.w_off;
  double *o0 = db + rw.out0;
  double *o1 = rw.out1 >= 0 ? db + rw.out1 : nullptr;
  const bool delta = rw.kind == ROW_DELTA;
  const bool lap = rw.comp == 1;  // biharmonic second component: w_c1 Lap phi and w_f1 d Lap phi/dn
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    const double4 c = fc[j];
    const double t = tanh_half(fma(c.x, rw.x, fma(c.y, rw.y, c.z)), s_exp2);
    const double s1 = fma(-t, t, 1.0);
    // Lap phi = |w|^2 tanh''(z) = -2 |w|^2 t (1 - t^2)  (c.w = 2 |w|^2)
    const double v = lap ? w_c1 * (-(c.w * t) * s1) : t;
    o0[j] = v;
    if (o1) o1[j] = v;
    if (delta) {
      // d phi/dn = (w . n) tanh'(z); d Lap phi/dn = |w|^2 (w . n) tanh'''(z),
      // tanh''' = -2 (1 - t^2)(1 - 3 t^2)
      const double wn = rw.nx * w[2 * j] + rw.ny * w[2 * j + 1];
      const double f = lap ? w_f1 * (-(c.w * wn) * s1 * fma(-3.0 * t, t, 1.0)) : w_f0 * (wn * s1);
      db[rw.out2 + j] = f;
      db[rw.out3 + j] = f;
    }
  }
}

// Second pass: rows that combine first-pass rows of the same subdomain.
//   Delta row with the change of variables: phi(x) - alpha phi(x_a) - beta phi(x_b)
//   A_m corner row: sum over the two edges of the mean of F phi over the corner
//   and the e edge points (the corner's flux from its point value)
__global__ void __launch_bounds__(256) special_combine_kernel(const SpecialRow *__restrict__ rows,
                                                              const SubDev *__restrict__ subs,
                                                              double *__restrict__ db, long long o_w,
                                                              double w_f0, double w_f1) {
  const SpecialRow rw = rows[blockIdx.x];
  const bool tinv = rw.kind == ROW_DELTA && (rw.ca >= 0 || rw.cb >= 0);
  if (!tinv && rw.kind != ROW_AM) return;
  const SubDev d = subs[rw.sub];
  const double *w = db + o_w + 2 * d.w_off;
  const long long M = d.M;
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    if (tinv) {
      double v = db[rw.out0 + j];
      if (rw.ca >= 0) v -= rw.alpha * db[rw.ca + j];
      if (rw.cb >= 0) v -= rw.beta * db[rw.cb + j];
      db[rw.out0 + j] = v;
      db[rw.out1 + j] = v;
    } else {
      const double wx = w[2 * j], wy = w[2 * j + 1];
      const double tc = db[rw.ca + j];  // phi at the corner
      double sc = 1.0 - tc * tc;
      // the corner flux w_f0 d phi/dn or, for the biharmonic second component,
      // w_f1 d Lap phi/dn = w_f1 |w|^2 (w . n) tanh''', tanh''' = -2 (1 - t^2)(1 - 3 t^2)
      sc = rw.comp == 1 ? w_f1 * (-2.0 * fma(wx, wx, wy * wy) * sc * fma(-3.0 * tc, tc, 1.0)) : w_f0 * sc;
      double v = 0.0;
      for (int e = 0; e < 2; ++e) {
        const int ne = rw.am_e[e];
        double acc = (rw.am_n[e][0] * wx + rw.am_n[e][1] * wy) * sc;
        for (int k = 0; k < ne; ++k) acc += db[rw.am_f[e] + k * M + j];
        v += acc / double(ne + 1);
      }
      db[rw.out0 + j] = v;
    }
  }
}

// ---- s-derivatives of the features (the hidden-layer scale: w = s w_hat,
// b = s b_hat, so z = w . x + b = s z_hat and dz/ds = z / s).  With t = tanh z,
// s1 = 1 - t^2:  d phi/ds = s1 z/s;  for L phi = 2 |w|^2 t s1 (|w|^2 = s^2 |w_hat|^2)
// d/ds = 2 L phi / s + 2 |w|^2 s1 (1 - 3 t^2) z/s;  the diffusion rows subtract
// d/ds [(grad a . w) s1] = (grad a . w) s1 (1/s - 2 t z/s);  F phi = (w . n) s1
// gives d/ds = (w . n) s1 (1/s - 2 t z/s).  The derivative rows go to the value
// rows' offsets + dshift of the subdomain (the scale tables' layout).
__global__ void __launch_bounds__(256) interior_rows_ds_kernel(const SubDev *__restrict__ subs, int sub0,
                                                               double *__restrict__ db, long long o_w,
                                                               long long o_fc, long long o_exp2, long long o_xint,
                                                               long long o_aint, long long o_gaint, int op,
                                                               double inv_s) {
  __shared__ double s_exp2[256];
  const SubDev d = subs[sub0 + blockIdx.y];
  const int r0 = blockIdx.x * 8;
  if (r0 >= d.nI) return;
  load_exp2tab(s_exp2, db + o_exp2);
  const double *w = db + o_w + 2 * d.w_off;
  const double4 *fc = reinterpret_cast<const double4 *>(db + o_fc) + d.w_off;
  for (int rr = 0; rr < 8; ++rr) {
    const int r = r0 + rr;
    if (r >= d.nI) break;
    const long long pi = d.int_off + r;
    const double x = db[o_xint + 2 * pi], y = db[o_xint + 2 * pi + 1];
    double a = 1.0, ax = 0.0, ay = 0.0;
    if (op == DDELM_OP_DIFFUSION) {
      a = db[o_aint + pi];
      ax = db[o_gaint + 2 * pi];
      ay = db[o_gaint + 2 * pi + 1];
    }
    double *o0 = db + d.oK + d.dshift + (long long)r * d.M;
    double *o1 = db + d.oKb + d.dshift + (long long)r * d.M;
    for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
      const double4 c = fc[j];  // 2 w_x, 2 w_y, 2 b, 2 |w|^2
      const double u = fma(c.x, x, fma(c.y, y, c.z));
      const double t = tanh_half(u, s_exp2);
      const double s1 = fma(-t, t, 1.0);
      const double zs = 0.5 * u * inv_s;       // z / s
      const double lp = (c.w * t) * s1;        // L phi (Poisson)
      double v = fma(2.0 * inv_s, lp, c.w * s1 * fma(-3.0 * t, t, 1.0) * zs);
      if (op == DDELM_OP_DIFFUSION) {
        const double ga = ax * w[2 * j] + ay * w[2 * j + 1];
        v = a * v - ga * s1 * fma(-2.0 * t, zs, inv_s);
      }
      o0[j] = v;
      o1[j] = v;
    }
  }
}

__global__ void __launch_bounds__(256) special_rows_ds_kernel(const SpecialRow *__restrict__ rows,
                                                              const SubDev *__restrict__ subs,
                                                              double *__restrict__ db, long long o_w,
                                                              long long o_fc, long long o_exp2, double inv_s) {
  __shared__ double s_exp2[256];
  const SpecialRow rw = rows[blockIdx.x];
  if (rw.kind == ROW_AM) return;
  load_exp2tab(s_exp2, db + o_exp2);
  const SubDev d = subs[rw.sub];
  const double *w = db + o_w + 2 * d.w_off;
  const double4 *fc = reinterpret_cast<const double4 *>(db + o_fc) + d.w_off;
  const long long sh = d.dshift;
  double *o0 = db + rw.out0 + sh;
  double *o1 = rw.out1 >= 0 ? db + rw.out1 + sh : nullptr;
  const bool delta = rw.kind == ROW_DELTA;
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    const double4 c = fc[j];
    const double u = fma(c.x, rw.x, fma(c.y, rw.y, c.z));
    const double t = tanh_half(u, s_exp2);
    const double s1 = fma(-t, t, 1.0);
    const double zs = 0.5 * u * inv_s;
    const double dp = s1 * zs;
    o0[j] = dp;
    if (o1) o1[j] = dp;
    if (delta) {
      const double f = (rw.nx * w[2 * j] + rw.ny * w[2 * j + 1]) * s1 * fma(-2.0 * t, zs, inv_s);
      db[rw.out2 + sh + j] = f;
      db[rw.out3 + sh + j] = f;
    }
  }
}

// Second pass on the derivative rows: the change-of-variables rows are the same
// combination of derivative rows; the A_m corner row's corner flux
// (w . n)(1 - t_c^2) has the derivative (w . n)(s1_c / s - 2 t_c dt_c/ds), with
// t_c from the value block and dt_c/ds from the derivative block.
__global__ void __launch_bounds__(256) special_combine_ds_kernel(const SpecialRow *__restrict__ rows,
                                                                 const SubDev *__restrict__ subs,
                                                                 double *__restrict__ db, long long o_w,
                                                                 double inv_s) {
  const SpecialRow rw = rows[blockIdx.x];
  const bool tinv = rw.kind == ROW_DELTA && (rw.ca >= 0 || rw.cb >= 0);
  if (!tinv && rw.kind != ROW_AM) return;
  const SubDev d = subs[rw.sub];
  const double *w = db + o_w + 2 * d.w_off;
  const long long M = d.M, sh = d.dshift;
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    if (tinv) {
      double v = db[rw.out0 + sh + j];
      if (rw.ca >= 0) v -= rw.alpha * db[rw.ca + sh + j];
      if (rw.cb >= 0) v -= rw.beta * db[rw.cb + sh + j];
      db[rw.out0 + sh + j] = v;
      db[rw.out1 + sh + j] = v;
    } else {
      const double wx = w[2 * j], wy = w[2 * j + 1];
      const double tc = db[rw.ca + j], dtc = db[rw.ca + sh + j];
      const double sc = 1.0 - tc * tc;
      double v = 0.0;
      for (int e = 0; e < 2; ++e) {
        const int ne = rw.am_e[e];
        double acc = (rw.am_n[e][0] * wx + rw.am_n[e][1] * wy) * fma(sc, inv_s, -2.0 * tc * dtc);
        for (int k = 0; k < ne; ++k) acc += db[rw.am_f[e] + sh + k * M + j];
        v += acc / double(ne + 1);
      }
      db[rw.out0 + sh + j] = v;
    }
  }
}

}  // namespace

// The scale gradient's local matrices of wave w: K_c, K-bar, A_m, A-bar and the
// evaluation matrix re-assembled into the scale buffers, then their s-derivatives.
cudaError_t launch_scale_features(const Plan &p, void *ws, int wave, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_ssubs);
  const SpecialRow *rows = reinterpret_cast<const SpecialRow *>(base + p.off_srows);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  const int s0 = wave * p.wave, s1 = std::min(p.n_sub, s0 + p.wave);
  int max_nI = 0;
  for (int i = s0; i < s1; ++i) max_nI = std::max(max_nI, p.subs[i].nI);
  const int r0 = p.wave_row0[wave], r1 = p.wave_row0[wave + 1];
  const int e0 = p.wave_erow0[wave], e1 = p.wave_erow0[wave + 1];
  const dim3 grid((max_nI + 7) / 8, s1 - s0);
  if (max_nI > 0) { interior_rows_kernel<<<grid, 256, 0, s>>>(subs, s0, db, p.o_w, p.o_fc, p.o_exp2, p.o_xint, p.o_aint, p.o_gaint, p.op, p.w_int); DDELM_COUNT_LAUNCH(); }
  if (r1 > r0) {
    { special_rows_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.w_c1, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
    { special_combine_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
  }
  if (e1 > e0) { special_rows_kernel<<<(unsigned)(e1 - e0), 256, 0, s>>>(rows + e0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.w_c1, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
  if (max_nI > 0) { interior_rows_ds_kernel<<<grid, 256, 0, s>>>(subs, s0, db, p.o_w, p.o_fc, p.o_exp2, p.o_xint, p.o_aint, p.o_gaint, p.op, p.inv_scale); DDELM_COUNT_LAUNCH(); }
  if (r1 > r0) {
    { special_rows_ds_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.inv_scale); DDELM_COUNT_LAUNCH(); }
    { special_combine_ds_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.inv_scale); DDELM_COUNT_LAUNCH(); }
  }
  if (e1 > e0) { special_rows_ds_kernel<<<(unsigned)(e1 - e0), 256, 0, s>>>(rows + e0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.inv_scale); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

// Features of the subdomains of one setup wave (their special rows included);
// wave 0 also writes the evaluation rows.
cudaError_t launch_features(const Plan &p, void *ws, int wave, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  const SpecialRow *rows = reinterpret_cast<const SpecialRow *>(base + p.off_rows);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  const int s0 = wave * p.wave, s1 = std::min(p.n_sub, s0 + p.wave);
  int max_nI = 0;
  for (int i = s0; i < s1; ++i) max_nI = std::max(max_nI, p.subs[i].nI);
  if (max_nI > 0) {
    dim3 grid((max_nI + 7) / 8, s1 - s0);
    { interior_rows_kernel<<<grid, 256, 0, s>>>(subs, s0, db, p.o_w, p.o_fc, p.o_exp2, p.o_xint, p.o_aint, p.o_gaint, p.op, p.w_int); DDELM_COUNT_LAUNCH(); }
  }
  const int r0 = p.wave_row0[wave], r1 = p.wave_row0[wave + 1];
  if (r1 > r0) {
    { special_rows_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.w_c1, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
    { special_combine_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
  }
  const int e0 = p.wave_row0[p.n_waves], e1 = int(p.rows.size());
  if (wave == 0 && e1 > e0) { special_rows_kernel<<<(unsigned)(e1 - e0), 256, 0, s>>>(rows + e0, subs, db, p.o_w, p.o_fc, p.o_exp2, p.w_c1, p.w_f0, p.w_f1); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

}  // namespace ddelm
