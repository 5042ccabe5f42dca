// Fused feature assembly (Sec. 2.2 and Sec. 2.2.1, Sec. 3.1, Sec. 3.2):
// phi_j(x) = tanh(w_j . x + b_j) and the rows of K_c^i, K-bar^i, A_m^i,
// A-bar^i and the evaluation matrix, written once in FP64 with coalesced
// row-major stores (consecutive threads -> consecutive neurons j).
//
//   L phi (Poisson)   = 2 |w|^2 t (1 - t^2)
//   L phi (diffusion) = 2 a |w|^2 t (1 - t^2) - (grad a . w)(1 - t^2)
//   B phi = C phi = t,   F phi = (w . n)(1 - t^2)
// with t = tanh(w . x + b).  The interior rows and the first pass over the
// other rows take one tanh per (point, neuron); the rows that combine point
// values or fluxes (change of variables, A_m corner rows) are formed from them.
#include <algorithm>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

__device__ __forceinline__ double feat_t(double wx, double wy, double b, double x, double y) {
  return tanh(fma(wx, x, wy * y) + b);
}

// Interior collocation rows: rows [0, nI) of K_c^i and K-bar^i.
__global__ void __launch_bounds__(256) interior_rows_kernel(const SubDev *__restrict__ subs, int sub0,
                                                            double *__restrict__ db, long long o_w,
                                                            long long o_b, long long o_xint,
                                                            long long o_aint, long long o_gaint, int op) {
  const SubDev d = subs[sub0 + blockIdx.y];
  const int r0 = blockIdx.x * 8;
  if (r0 >= d.nI) return;
  const double *w = db + o_w + 2 * d.w_off;
  const double *b = db + o_b + d.w_off;
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
      const double wx = w[2 * j], wy = w[2 * j + 1];
      const double t = feat_t(wx, wy, b[j], x, y);
      const double s1 = 1.0 - t * t;
      const double w2 = wx * wx + wy * wy;
      double v = 2.0 * w2 * t * s1;
      if (op == DDELM_OP_DIFFUSION) v = a * v - (ax * wx + ay * wy) * s1;
      o0[j] = v;
      o1[j] = v;
    }
  }
}

// First pass over the special rows: one tanh per (point, neuron).
__global__ void __launch_bounds__(256) special_rows_kernel(const SpecialRow *__restrict__ rows,
                                                           const SubDev *__restrict__ subs,
                                                           double *__restrict__ db, long long o_w,
                                                           long long o_b) {
  const SpecialRow rw = rows[blockIdx.x];
  if (rw.kind == ROW_AM) return;
  const SubDev d = subs[rw.sub];
  const double *w = db + o_w + 2 * d.w_off;
  const double *b = db + o_b + d.w_off;
  double *o0 = db + rw.out0;
  double *o1 = rw.out1 >= 0 ? db + rw.out1 : nullptr;
  const bool delta = rw.kind == ROW_DELTA;
  for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
    const double wx = w[2 * j], wy = w[2 * j + 1];
    const double t = feat_t(wx, wy, b[j], rw.x, rw.y);
    o0[j] = t;
    if (o1) o1[j] = t;
    if (delta) {
      const double f = (rw.nx * wx + rw.ny * wy) * (1.0 - t * t);
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
                                                              double *__restrict__ db, long long o_w) {
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
      const double tc = db[rw.ca + j];
      const double sc = 1.0 - tc * tc;
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

}  // namespace

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
    { interior_rows_kernel<<<grid, 256, 0, s>>>(subs, s0, db, p.o_w, p.o_b, p.o_xint, p.o_aint, p.o_gaint, p.op); DDELM_COUNT_LAUNCH(); }
  }
  const int r0 = p.wave_row0[wave], r1 = p.wave_row0[wave + 1];
  if (r1 > r0) {
    { special_rows_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w, p.o_b); DDELM_COUNT_LAUNCH(); }
    { special_combine_kernel<<<(unsigned)(r1 - r0), 256, 0, s>>>(rows + r0, subs, db, p.o_w); DDELM_COUNT_LAUNCH(); }
  }
  const int e0 = p.wave_row0[p.n_waves], e1 = int(p.rows.size());
  if (wave == 0 && e1 > e0) { special_rows_kernel<<<(unsigned)(e1 - e0), 256, 0, s>>>(rows + e0, subs, db, p.o_w, p.o_b); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

}  // namespace ddelm
