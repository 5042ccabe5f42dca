// Batched Cholesky factorisation with explicit triangular inverse (one CTA
// per matrix) in FP64 or FP32, the small matrix operations of the polished
// FP32 scheme, the coarse-matrix assembly of Sec. 3 (S_Pi assembled in full),
// and small helpers (identity fill, right-hand-side gather).
//
// A Cholesky pass of shifted CholeskyQR on [K; eps I] factors
// G + (eps^2 + s) I:
//   ridge passes (the first): eps^2 = eps_rel^2 tr(G)/M is the ridge of the
//     local least-squares problem and Z = eps R^{-1} the ridge block of the
//     first Q;
//   shift kind 1 (FP64 first pass): s = shift_rel tr(G + eps^2 I) with
//     shift_rel = 11 ((m+M) M + M (M+1)) u, u = 2^-53 (raised to cover the
//     slice truncation of a tensor-core Gram);
//   shift kind 2 (FP32 passes): s = shift_rel max diag(G + eps^2 I).
// A pivot that is not positive marks the matrix in the status array; the
// factorisation continues with a unit pivot so that no NaN propagates.
#include <algorithm>

#include "ddelm_internal.h"

namespace ddelm {

namespace {

constexpr int CT = 512;
constexpr int NB = 16;   // panel rows

__device__ __forceinline__ double shfl_xor(unsigned m, double v, int o) { return __shfl_xor_sync(m, v, o); }
__device__ __forceinline__ float shfl_xor(unsigned m, float v, int o) { return __shfl_xor_sync(m, v, o); }

}  // namespace

// Double-FP32 numbers x = hi + lo with |lo| <= ulp(hi)/2: about 46 significant
// bits carried by the FP32 pipe, which this GPU runs at 64 times its FP64 rate.
// Built from Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based exact
// product (a b = p + e with e = fma(a, b, -p)); additions renormalise once, so
// a sum is accurate to about 2^-47 of |x| + |y| (backward stable, like an FP64
// addition at that unit roundoff), which is all a Cholesky factorisation needs.
// The functions live in their own namespace and are found by argument-dependent
// lookup, so the FP64 and FP32 instances of the factorisation are unchanged.
namespace dw {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ ff(float h) : hi(h), lo(0.0f) {}
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = a + b;
  return ff(s, b - (s - a));
}
__device__ __forceinline__ ff operator+(ff x, ff y) {
  const ff s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ ff operator-(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff &operator+=(ff &x, ff y) { return x = x + y; }
__device__ __forceinline__ ff &operator-=(ff &x, ff y) { return x = x - y; }
// product: exact product of the high parts plus the cross terms (lo lo dropped)
__device__ __forceinline__ ff operator*(ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
// a b + c with one renormalisation
__device__ __forceinline__ ff fma(ff a, ff b, ff c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const ff s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, s.lo + (e + c.lo));
}
// 1 / x: the FP32 reciprocal and one Newton step r + r (1 - x r)
__device__ __forceinline__ ff recip(ff x) {
  const ff r(1.0f / x.hi);
  return fma(r, fma(-x, r, ff(1.0f)), r);
}
__device__ __forceinline__ ff operator/(ff a, ff b) { return a * recip(b); }
// sqrt(a): the FP32 root y and one correction (a - y^2) / (2 y), y^2 exact by FMA
__device__ __forceinline__ ff sqrt(ff a) {
  const float y = sqrtf(a.hi);
  if (!(y > 0.0f)) return ff(y);
  return fast_two_sum(y, (fmaf(-y, y, a.hi) + a.lo) / (2.0f * y));
}
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool isfinite(ff a) { return ::isfinite(a.hi) && ::isfinite(a.lo); }
__device__ __forceinline__ ff shfl_xor(unsigned m, ff v, int o) {
  return ff(__shfl_xor_sync(m, v.hi, o), __shfl_xor_sync(m, v.lo, o));
}
__device__ __forceinline__ ff from_double(double d) {
  const float h = float(d);
  return ff(h, float(d - double(h)));
}
__device__ __forceinline__ double to_double(ff x) { return double(x.hi) + double(x.lo); }

}  // namespace dw

namespace {

// Blocked right-looking upper Cholesky A = R^T R in place (upper triangle), then
// V = R^{-1} by blocked back substitution, in precision T.  The panel (NB rows
// of the trailing matrix) lives in shared memory; the trailing update is a
// register-tiled SYRK (4x4 tiles per thread), so A is read and written once per
// panel.  band > 0: A (and R) vanish beyond band superdiagonals, and only
// in-band entries are touched.  A non-positive pivot sets *bad and continues
// with a unit pivot.
template <typename T>
__device__ void chol_inv_core(T *A, T *V, int M, int band, T *P, int *bad, int invb = 0, int ld = 0) {
  if (ld <= 0) ld = M;  // A and V: M x M blocks with leading dimension ld
  __shared__ T s_piv, s_rinv;
  __shared__ T rinv[NB];
  const int tid = threadIdx.x;
  const int BW = band > 0 ? band : M;
  for (int k0 = 0; k0 < M; k0 += NB) {
    const int nb = min(NB, M - k0);
    const int W = min(M, k0 + nb + BW) - k0;  // panel columns k0 .. k0+W
    for (int e = tid; e < nb * W; e += CT) {
      const int r = e / W, c = e % W;
      P[r * W + c] = A[(long long)(k0 + r) * ld + k0 + c];
    }
    __syncthreads();
    for (int t = 0; t < nb; ++t) {  // unblocked elimination inside the panel
      if (tid == 0) {
        T piv = P[t * W + t];
        if (!(piv > T(0)) || !isfinite(piv)) {
          *bad = 1;
          piv = T(1);
        }
        s_piv = sqrt(piv);
        s_rinv = T(1) / s_piv;
      }
      __syncthreads();
      const T r = s_piv, ri = s_rinv;
      for (int c = t + tid; c < W; c += CT) P[t * W + c] = c == t ? r : P[t * W + c] * ri;
      __syncthreads();
      for (int e = tid; e < (nb - t - 1) * W; e += CT) {
        const int u = t + 1 + e / W, c = e % W;
        if (c >= u) P[u * W + c] = fma(-P[t * W + u], P[t * W + c], P[u * W + c]);
      }
      __syncthreads();
    }
    for (int e = tid; e < nb * W; e += CT) {
      const int r = e / W, c = e % W;
      if (c >= r) A[(long long)(k0 + r) * ld + k0 + c] = P[r * W + c];
    }
    // trailing update of the upper triangle: A[i][j] -= sum_t P[t][i] P[t][j], i <= j
    const int T0 = k0 + nb, T1 = k0 + W, nt = T1 - T0;  // only columns the panel reaches
    if (nt > 0) {
      const int nbt = (nt + 3) / 4;
      const int ntiles = nbt * (nbt + 1) / 2;
      for (int q = tid; q < ntiles; q += CT) {
        // tile row bi: the largest b with S(b) = b nbt - b (b - 1) / 2 <= q (the
        // tiles before row b), from the root of the quadratic, corrected to the
        // exact integer (a linear search cost as much as the tile at M = 1000)
        const int tw = 2 * nbt + 1;
        int bi = (int)(0.5f * ((float)tw - sqrtf((float)(tw * tw - 8 * q))));
        bi = max(0, min(bi, nbt - 1));
        while (bi > 0 && bi * nbt - bi * (bi - 1) / 2 > q) --bi;
        while (bi + 1 < nbt && (bi + 1) * nbt - (bi + 1) * bi / 2 <= q) ++bi;
        const int rem = q - (bi * nbt - bi * (bi - 1) / 2);
        const int bj = bi + rem;
        const int i0 = T0 + 4 * bi, j0 = T0 + 4 * bj;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int t = 0; t < nb; ++t) {
          T pa[4], pb[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) pa[a] = (i0 + a < T1) ? P[t * W + (i0 + a - k0)] : T(0);
#pragma unroll
          for (int b = 0; b < 4; ++b) pb[b] = (j0 + b < T1) ? P[t * W + (j0 + b - k0)] : T(0);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(pa[a], pb[b], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int i = i0 + a;
          if (i >= T1) continue;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int j = j0 + b;
            if (j < T1 && j >= i) A[(long long)i * ld + j] -= acc[a][b];
          }
        }
      }
    }
    __syncthreads();
  }
  // V = R^{-1}: block rows from the bottom;
  // V[i][j] = (delta_ij - sum_{k>i} R[i][k] V[k][j]) / R[i][i], j >= i
  for (long long e = tid; e < (long long)M * M; e += CT) V[(e / M) * ld + e % M] = T(0);
  __syncthreads();
  const int nblk = (M + NB - 1) / NB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int i0 = b * NB, nb = min(NB, M - i0), i1 = i0 + nb;
    const int W = min(M, i0 + nb + BW) - i0;  // R[i0..i1][i0 .. i0+W] holds the block's nonzeros
    for (int e = tid; e < nb * W; e += CT) {
      const int r = e / W, c = e % W;
      P[r * W + c] = A[(long long)(i0 + r) * ld + i0 + c];
    }
    if (tid < nb) rinv[tid] = T(1) / A[(long long)(i0 + tid) * ld + i0 + tid];
    __syncthreads();
    // tpc consecutive lanes share a column (strided k), so that the short block
    // rows near the bottom still keep every warp busy.  invb > 0: columns only
    // up to the end of the invb-block holding row i0 (diagonal blocks of R^{-1})
    const int ncol = (invb > 0 ? min(M, (i0 / invb + 1) * invb) : M) - i0;
    int tpc = 1;
    while (tpc < 16 && ncol * tpc * 2 <= CT) tpc *= 2;
    const int part = tid % tpc;
    for (int jj = tid / tpc; jj < ncol; jj += CT / tpc) {
      const int j = i0 + jj;
      T acc[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) acc[r] = T(0);
      const int kend = min(j, i0 + W - 1);
      // eight loads of V in flight per thread before their FMAs (one at a time
      // the loop waited an L2 round trip per k); the same accumulation order
      int k = i1 + part;
      for (; k + 7 * tpc <= kend; k += 8 * tpc) {
        T vk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) vk[u] = V[(long long)(k + u * tpc) * ld + j];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int r = 0; r < NB; ++r) acc[r] = fma(P[r * W + (k + u * tpc - i0)], vk[u], acc[r]);
      }
      for (; k <= kend; k += tpc) {
        const T vk = V[(long long)k * ld + j];
#pragma unroll
        for (int r = 0; r < NB; ++r) acc[r] = fma(P[r * W + (k - i0)], vk, acc[r]);
      }
      if (tpc > 1) {
        // the tpc lanes of this column: aligned, inside one warp, same iteration
        const unsigned gmask = ((tpc == 32) ? 0xffffffffu : ((1u << tpc) - 1u)) << ((tid & 31) & ~(tpc - 1));
        __syncwarp(gmask);
        for (int o = 1; o < tpc; o <<= 1)
#pragma unroll
          for (int r = 0; r < NB; ++r) acc[r] += shfl_xor(gmask, acc[r], o);
      }
      if (part == 0) {
      T x[NB];
#pragma unroll
      for (int r = NB - 1; r >= 0; --r) {
        if (r >= nb) {
          x[r] = T(0);
          continue;
        }
        const int i = i0 + r;
        T v = (j == i ? T(1) : T(0)) - acc[r];
#pragma unroll
        for (int u = r + 1; u < NB; ++u)
          if (u < nb) v = fma(-P[r * W + u], x[u], v);
        x[r] = (j >= i) ? v * rinv[r] : T(0);
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb && j >= i0 + r) V[(long long)(i0 + r) * ld + j] = x[r];
      }
    }
    __syncthreads();
  }
}

// trace and maximum of the diagonal of an FP64 matrix (block reduction)
__device__ void diag_stats(const double *G, int M, double *tr_out, double *mx_out) {
  __shared__ double rt[CT / 32], rm[CT / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double t = 0.0, mx = 0.0;
  for (int j = tid; j < M; j += CT) {
    const double g = G[(long long)j * M + j];
    t += g;
    mx = fmax(mx, g);
  }
  for (int o = 16; o > 0; o >>= 1) {
    t += __shfl_xor_sync(0xffffffffu, t, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    rt[wid] = t;
    rm[wid] = mx;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < CT / 32; ++k) {
      a += rt[k];
      b = fmax(b, rm[k]);
    }
    *tr_out = a;
    *mx_out = b;
  }
  __syncthreads();
}

// The diagonal additions of a Cholesky pass: the ridge eps^2 = eps_rel^2 tr/M
// (ridge passes) and the stabilising shift (shift_rel * tr(G + eps^2 I) for
// shift kind 1, shift_rel * max diag(G + eps^2 I) for kind 2).
__device__ void diag_additions(const CholDesc &cd, const double *G, double *eps2_out, double *add_out) {
  __shared__ double s_tr, s_mx;
  diag_stats(G, cd.M, &s_tr, &s_mx);
  const double eps2 = cd.ridge ? cd.eps_rel * cd.eps_rel * s_tr / double(cd.M) : 0.0;
  double shift = 0.0;
  if (cd.shift_kind == 1) shift = cd.shift_rel * (s_tr + cd.M * eps2);
  if (cd.shift_kind == 2) shift = cd.shift_rel * (s_mx + eps2);
  *eps2_out = eps2;
  *add_out = eps2 + shift;
}

// FP64 pass: factor in place in G, V = R^{-1}.  mode 1 (the first step of a
// blocked factorisation, whose diagonal blocks are then factored by mode 0
// with a leading dimension and its panels and trailing updates are
// tensor-core GEMMs): only the diagonal additions, eps, and V zeroed.
__global__ void __launch_bounds__(CT) chol_inv_kernel(const CholDesc *__restrict__ descs,
                                                      double *__restrict__ db, int *__restrict__ status) {
  extern __shared__ double P[];
  const CholDesc cd = descs[blockIdx.x];
  const int M = cd.M;
  const int ld = cd.ld > 0 ? cd.ld : M;
  double *G = db + cd.g;
  double *V = db + cd.v;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  double eps2 = 0.0, add = 0.0;
  if (cd.mode == 1 || cd.ridge || cd.shift_kind) diag_additions(cd, G, &eps2, &add);
  if (add != 0.0) {
    for (int j = threadIdx.x; j < M; j += CT) G[(long long)j * ld + j] += add;
    __syncthreads();
  }
  if (cd.epsout >= 0 && threadIdx.x == 0) db[cd.epsout] = sqrt(eps2);
  if (cd.mode == 1) {
    for (long long e = threadIdx.x; e < (long long)M * M; e += CT) V[e] = 0.0;
    return;
  }
  chol_inv_core<double>(G, V, M, cd.band, P, &s_bad, cd.inv_block, ld);
  if (cd.z >= 0) {
    double *Z = db + cd.z;
    const double e = sqrt(eps2);
    for (long long q = threadIdx.x; q < (long long)M * M; q += CT) Z[q] = e * V[q];
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_bad) status[cd.status] = 1;
}

// FP32 pass (a preconditioning factor of shifted CholeskyQR: every product
// with V is exact downstream, so V need only be well conditioned): G is read
// in FP64, factored in FP32 in the work buffer w (2 M^2 floats), V written in
// FP64.
__global__ void __launch_bounds__(CT) chol_inv32_kernel(const CholDesc *__restrict__ descs,
                                                        double *__restrict__ db, int *__restrict__ status) {
  extern __shared__ float P32[];
  const CholDesc cd = descs[blockIdx.x];
  const int M = cd.M;
  const double *G = db + cd.g;
  double *V = db + cd.v;
  float *A = reinterpret_cast<float *>(db + cd.w);
  float *V32 = A + (long long)M * M;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  double eps2 = 0.0, add = 0.0;
  diag_additions(cd, G, &eps2, &add);
  for (long long e = threadIdx.x; e < (long long)M * M; e += CT) {
    const int i = int(e / M), j = int(e % M);
    A[e] = j >= i ? float(G[e] + (i == j ? add : 0.0)) : 0.0f;
  }
  __syncthreads();
  chol_inv_core<float>(A, V32, M, 0, P32, &s_bad);
  const double ez = sqrt(eps2);
  for (long long e = threadIdx.x; e < (long long)M * M; e += CT) {
    const double v = double(V32[e]);
    V[e] = v;
    if (cd.z >= 0) db[cd.z + e] = ez * v;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_bad) status[cd.status] = 1;
}

// Double-FP32 pass (a preconditioning factor of shifted CholeskyQR, as the FP32
// pass, in about 46-bit arithmetic so that two passes suffice): G + (eps^2 + s) I
// is converted in place to double-FP32 numbers (8 bytes, like the FP64 entries
// they replace), factored, and R (upper triangle of G) and V = R^{-1} are
// converted back to FP64 in place.
__global__ void __launch_bounds__(CT) chol_inv_dw_kernel(const CholDesc *__restrict__ descs,
                                                         double *__restrict__ db, int *__restrict__ status) {
  extern __shared__ dw::ff Pw[];
  const CholDesc cd = descs[blockIdx.x];
  const int M = cd.M;
  double *G = db + cd.g;
  double *V = db + cd.v;
  dw::ff *A = reinterpret_cast<dw::ff *>(G);
  dw::ff *Vw = reinterpret_cast<dw::ff *>(V);
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  double eps2 = 0.0, add = 0.0;
  diag_additions(cd, G, &eps2, &add);
  // the factorisation reads the upper triangle only: convert that (the FP64
  // conversions run on this GPU's slow FP64 pipe) and zero the rest
  for (long long e = threadIdx.x; e < (long long)M * M; e += CT) {
    const long long i = e / M, j = e % M;
    A[e] = j >= i ? dw::from_double(G[e] + (i == j ? add : 0.0)) : dw::ff(0.0f);  // own entries only
  }
  __syncthreads();
  if (cd.epsout >= 0 && threadIdx.x == 0) db[cd.epsout] = sqrt(eps2);
  chol_inv_core<dw::ff>(A, Vw, M, cd.band, Pw, &s_bad, cd.inv_block);
  __syncthreads();
  const double ez = sqrt(eps2);
  for (long long e = threadIdx.x; e < (long long)M * M; e += CT) {
    const bool up = e % M >= e / M;  // R and V are upper triangular
    G[e] = up ? dw::to_double(A[e]) : 0.0;
    const double v = up ? dw::to_double(Vw[e]) : 0.0;
    V[e] = v;
    if (cd.z >= 0) db[cd.z + e] = ez * v;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_bad) status[cd.status] = 1;
}

// FP32 copies of the operators the inner CG of MIXED precision applies
__global__ void convert_f32_kernel(const ConvSeg *__restrict__ segs, const double *__restrict__ db,
                                   float *__restrict__ fb) {
  const ConvSeg sg = segs[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < sg.n; e += (long long)gridDim.x * blockDim.x)
    fb[sg.dst + e] = (float)db[sg.src + e];
}

// small batched matrix operations of the polishing step:
//   op 0: C = -I ;  op 1: C = I - A/2 + 3/8 B - 5/16 D  (the series of
//   (I + A)^{-1/2} with B = A^2, D = A^3) ;  op 2: C symmetric from its upper
//   triangle ;  op 3: C = A ;  op 4: C = A - I ;  op 5: C = b A (b a scalar in memory).
// op 1 flags the subdomain when max |A| > 1e-4: beyond that the neglected
// fourth-order term could reach the FP64 level.
__global__ void matop_kernel(const MatopDesc *__restrict__ descs, double *__restrict__ db, int *__restrict__ status) {
  const MatopDesc md = descs[blockIdx.y];
  const long long n = (long long)md.M * md.M;
  bool big = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / md.M, j = e % md.M;
    if (md.op == 0) {
      db[md.c + e] = i == j ? -1.0 : 0.0;
    } else if (md.op == 1) {
      const double a = db[md.a + e];
      big |= !(fabs(a) <= 1e-4);
      double w = (i == j ? 1.0 : 0.0) - 0.5 * a + 0.375 * db[md.b + e];
      if (md.d >= 0) w -= 0.3125 * db[md.d + e];
      db[md.c + e] = w;
    } else if (md.op == 2) {
      if (i > j) db[md.c + e] = db[md.c + j * md.M + i];
    } else if (md.op == 3) {
      db[md.c + e] = db[md.a + e];
    } else if (md.op == 4) {
      db[md.c + e] = db[md.a + e] - (i == j ? 1.0 : 0.0);
    } else {
      db[md.c + e] = db[md.b] * db[md.a + e];
    }
  }
  if (big) status[md.status] = 1;
}

// Sec. 3: D_PiPi = sum_i R_Pi^T Lambda_PiPi^i R_Pi and the first two terms of
// S_Pi = sum_i R_Pi^T (I - Psi^i)_PiPi R_Pi (+ D_PiPi^T D_PiPi added by a GEMM).
// One CTA walks the subdomains in order, so the sums are deterministic.
// D_PiPi = sum_i R_Pi^T Lambda^i_PiPi R_Pi, S_Pi = sum_i R_Pi^T (I - Psi^i)_PiPi R_Pi:
// a thread per global entry (P, Q), summing over the subdomains that hold both
// corners in increasing subdomain order (the owner lists are in that order),
// onto the zeroed matrices
__global__ void coarse_assembly_kernel(const SubDev *__restrict__ subs, const int *__restrict__ ints,
                                       double *__restrict__ db, int n_pi, int o_pi_own, long long o_Dpp,
                                       long long o_Spi) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n_pi * n_pi;
       e += (long long)gridDim.x * blockDim.x) {
    const int P = int(e / n_pi), Q = int(e % n_pi);
    double ds = 0.0, ss = 0.0;
    for (int o = 0; o < 4; ++o) {
      const int sub = ints[o_pi_own + 8 * P + 2 * o];
      if (sub < 0) continue;
      const int a = ints[o_pi_own + 8 * P + 2 * o + 1];
      const SubDev &d = subs[sub];
      for (int b = 0; b < d.nPi; ++b)
        if (ints[d.gpi_off + b] == Q) {
          ds += db[d.oLam + (long long)a * d.nG + b];
          ss += (a == b ? 1.0 : 0.0) - db[d.oPsi + (long long)a * d.nG + b];
        }
    }
    db[o_Dpp + e] += ds;
    db[o_Spi + e] += ss;
  }
}

__global__ void fill_identity_kernel(double *dst, int n, double diag) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = (e / n == e % n) ? diag : 0.0;
}

// F^i = [w_int f(x_I); g(x_B)] per subdomain ([nI + nB] x R); the Dirichlet data
// of the second biharmonic component (global index >= nb0) times w_c1
__global__ void gather_rhs_kernel(const SubDev *__restrict__ subs, const int *__restrict__ ints,
                                  double *__restrict__ db, const double *__restrict__ f_int,
                                  const double *__restrict__ g_bnd, int R, double w_int, double w_c1, int nb0) {
  const SubDev d = subs[blockIdx.x];
  const int rows = d.nI + d.nB;
  double *F = db + d.oF;
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
    const int r = e / R, c = e % R;
    if (r < d.nI) {
      F[e] = w_int * f_int[(d.int_off + r) * R + c];
    } else {
      const int gb = ints[d.bnd_off + r - d.nI];
      F[e] = (gb >= nb0 ? w_c1 : 1.0) * g_bnd[(long long)gb * R + c];
    }
  }
}

// adjoint inputs per subdomain: C = dL/dc rows, U = dL/du rows (zero if absent)
__global__ void adjoint_init_kernel(const SubDev *__restrict__ subs, double *__restrict__ db,
                                    const double *__restrict__ grad_c, const double *__restrict__ grad_u, int R) {
  const SubDev d = subs[blockIdx.x];
  for (int e = threadIdx.x; e < d.M * R; e += blockDim.x) db[d.oC + e] = grad_c ? grad_c[d.w_off * R + e] : 0.0;
  for (int e = threadIdx.x; e < d.nE * R; e += blockDim.x) db[d.oU + e] = grad_u ? grad_u[d.eval_off * R + e] : 0.0;
}

__global__ void copy_c_to_y_kernel(const SubDev *__restrict__ subs, double *__restrict__ db, int R) {
  const SubDev d = subs[blockIdx.x];
  for (int e = threadIdx.x; e < d.M * R; e += blockDim.x) db[d.oY + e] = db[d.oC + e];
}

// dL/df = interior rows of F-bar; dL/dg = sum over the owners of each Dirichlet point
__global__ void adjoint_scatter_f_kernel(const SubDev *__restrict__ subs, const double *__restrict__ db,
                                         double *__restrict__ grad_f, int R, double w_int) {
  const SubDev d = subs[blockIdx.x];
  for (int e = threadIdx.x; e < d.nI * R; e += blockDim.x) grad_f[d.int_off * R + e] = w_int * db[d.oF + e];
}

__global__ void adjoint_scatter_g_kernel(const SubDev *__restrict__ subs, const int *__restrict__ ints,
                                         const double *__restrict__ db, double *__restrict__ grad_g, int n_bnd,
                                         int o_own, int R, double w_c1, int nb0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_bnd * R; e += gridDim.x * blockDim.x) {
    const int b = e / R, k = e % R;
    double v = 0.0;
    for (int o = 0; o < 2; ++o) {
      const int s = ints[o_own + 4 * b + 2 * o];
      if (s < 0) continue;
      const int r = ints[o_own + 4 * b + 2 * o + 1];
      const SubDev &d = subs[s];
      v += db[d.oF + (long long)(d.nI + r) * R + k];
    }
    grad_g[e] = (b >= nb0 ? w_c1 : 1.0) * v;
  }
}

}  // namespace

cudaError_t launch_adjoint_init(const Plan &p, void *ws, const double *grad_c, const double *grad_u, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  { adjoint_init_kernel<<<p.n_sub, 256, 0, s>>>(reinterpret_cast<const SubDev *>(base + p.off_subs),
                                              reinterpret_cast<double *>(base + p.off_dbl), grad_c, grad_u, p.n_rhs); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_copy_c_to_y(const Plan &p, void *ws, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  { copy_c_to_y_kernel<<<p.n_sub, 256, 0, s>>>(reinterpret_cast<const SubDev *>(base + p.off_subs),
                                             reinterpret_cast<double *>(base + p.off_dbl), p.n_rhs); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_scatter(const Plan &p, void *ws, double *grad_f, double *grad_g, cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  const double *db = reinterpret_cast<const double *>(base + p.off_dbl);
  if (grad_f && p.sz.sum_int > 0) { adjoint_scatter_f_kernel<<<p.n_sub, 256, 0, s>>>(subs, db, grad_f, p.n_rhs, p.w_int); DDELM_COUNT_LAUNCH(); }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (grad_g && p.sz.n_bnd > 0)
    { adjoint_scatter_g_kernel<<<64, 256, 0, s>>>(subs, reinterpret_cast<const int *>(base + p.off_ints), db, grad_g,
                                                p.sz.n_bnd, p.o_bnd_own, p.n_rhs, p.w_c1, p.nb0); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_chol_phase(const Plan &p, const CholPhase &ph, void *ws, cudaStream_t s) {
  if (ph.ndesc == 0) return cudaSuccess;
  char *base = static_cast<char *>(ws);
  const CholDesc *descs = reinterpret_cast<const CholDesc *>(base + p.off_cdesc) + ph.desc0;
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  int *status = reinterpret_cast<int *>(db + p.o_status);
  int maxM = 0;
  for (int k = 0; k < ph.ndesc; ++k) maxM = p.cdesc[ph.desc0 + k].M > maxM ? p.cdesc[ph.desc0 + k].M : maxM;
  const int prec = p.cdesc[ph.desc0].prec;  // one precision per phase
  const bool f32 = prec == 1, fdw = prec == 2;
  const size_t smem = (f32 ? sizeof(float) : sizeof(double)) * (size_t)NB * (size_t)maxM;  // double-FP32: 8 B
  if (smem > 48 * 1024) {
    cudaError_t e = f32   ? cudaFuncSetAttribute(chol_inv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                    : fdw ? cudaFuncSetAttribute(chol_inv_dw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                          : cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (f32)
    { chol_inv32_kernel<<<ph.ndesc, CT, smem, s>>>(descs, db, status); DDELM_COUNT_LAUNCH(); }
  else if (fdw)
    { chol_inv_dw_kernel<<<ph.ndesc, CT, smem, s>>>(descs, db, status); DDELM_COUNT_LAUNCH(); }
  else
    { chol_inv_kernel<<<ph.ndesc, CT, smem, s>>>(descs, db, status); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_matop_phase(const Plan &p, const MatopPhase &ph, void *ws, cudaStream_t s) {
  if (ph.ndesc == 0) return cudaSuccess;
  char *base = static_cast<char *>(ws);
  const MatopDesc *descs = reinterpret_cast<const MatopDesc *>(base + p.off_mdesc) + ph.desc0;
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  { matop_kernel<<<dim3(16, ph.ndesc), 256, 0, s>>>(descs, db, reinterpret_cast<int *>(db + p.o_status)); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_chol_table(const CholDesc *descs, int n, int maxM, double *db, int *status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * (size_t)NB * (size_t)maxM;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  { chol_inv_kernel<<<n, CT, smem, s>>>(descs, db, status); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_convert_f32(const Plan &p, void *ws, cudaStream_t s) {
  if (p.conv.empty()) return cudaSuccess;
  char *base = static_cast<char *>(ws);
  const ConvSeg *segs = reinterpret_cast<const ConvSeg *>(base + p.off_conv);
  const double *db = reinterpret_cast<const double *>(base + p.off_dbl);
  float *fb = reinterpret_cast<float *>(const_cast<double *>(db) + p.o_f32);
  { convert_f32_kernel<<<dim3(8, (unsigned)p.conv.size()), 256, 0, s>>>(segs, db, fb); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_coarse_assembly(const Plan &p, void *ws, cudaStream_t s) {
  if (p.n_pi == 0) return cudaSuccess;
  char *base = static_cast<char *>(ws);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  const int *ints = reinterpret_cast<const int *>(base + p.off_ints);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  const long long nn = (long long)p.n_pi * p.n_pi;
  const unsigned grid = (unsigned)std::min<long long>((nn + 255) / 256, 4096);
  { coarse_assembly_kernel<<<grid, 256, 0, s>>>(subs, ints, db, p.n_pi, p.o_pi_own, p.o_Dpp, p.o_Spi); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_fill_identity(double *dst, int n, double diag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  { fill_identity_kernel<<<64, 256, 0, s>>>(dst, n, diag); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

cudaError_t launch_gather_rhs(const Plan &p, void *ws, const double *f_int, const double *g_bnd,
                              cudaStream_t s) {
  char *base = static_cast<char *>(ws);
  const SubDev *subs = reinterpret_cast<const SubDev *>(base + p.off_subs);
  const int *ints = reinterpret_cast<const int *>(base + p.off_ints);
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  { gather_rhs_kernel<<<p.n_sub, 256, 0, s>>>(subs, ints, db, f_int, g_bnd, p.n_rhs, p.w_int, p.w_c1, p.nb0);
    DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

}  // namespace ddelm
