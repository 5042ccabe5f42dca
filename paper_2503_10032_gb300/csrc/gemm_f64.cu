// Batched FP64 GEMM engine: C = alpha op(A) op(B) + beta C over a flat list
// of square output tiles (64 x 64, or 16 x 16 for tiny products such as a
// small coarse space, which then spread over more SMs) drawn from any number
// of descriptors of any shapes (uneven subdomains are just more descriptors).
// Triangular operands are flagged so that the k loop skips the zero blocks.
// FP64 runs on the CUDA cores (DFMA); each thread owns a (T/16) x (T/16)
// register tile, operands are staged in shared memory in 16-deep k slices
// with a double buffer.
#include "ddelm_internal.h"

namespace ddelm {

namespace {

constexpr int BK = 16, NT = 256;

template <int BM>
__device__ __forceinline__ void load_tiles(const double *__restrict__ A, const double *__restrict__ B,
                                           const GemmDesc &d, int m0, int n0, int k0, int kbeg, int kend,
                                           double (*As)[BM + 1], double (*Bs)[BM + 1]) {
  constexpr int BN = BM;
  const int tid = threadIdx.x;
#pragma unroll
  for (int t = 0; t < (BM * BK) / NT; ++t) {
    const int e = tid + t * NT;
    int i, kk;
    if (!d.ta) {
      i = e / BK;
      kk = e % BK;
    } else {
      i = e % BM;
      kk = e / BM;
    }
    const int gi = m0 + i, gk = k0 + kk;
    double v = 0.0;
    if (gi < d.m && gk >= kbeg && gk < kend) v = d.ta ? A[(long long)gk * d.lda + gi] : A[(long long)gi * d.lda + gk];
    As[kk][i] = v;
  }
#pragma unroll
  for (int t = 0; t < (BN * BK) / NT; ++t) {
    const int e = tid + t * NT;
    int j, kk;
    if (!d.tb) {
      j = e % BN;
      kk = e / BN;
    } else {
      kk = e % BK;
      j = e / BK;
    }
    const int gj = n0 + j, gk = k0 + kk;
    double v = 0.0;
    if (gj < d.n && gk >= kbeg && gk < kend) v = d.tb ? B[(long long)gj * d.ldb + gk] : B[(long long)gk * d.ldb + gj];
    Bs[kk][j] = v;
  }
}

template <int BM>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(const GemmDesc *__restrict__ descs,
                                                      const GemmTile *__restrict__ tiles,
                                                      double *__restrict__ db) {
  constexpr int BN = BM, RT = BM / 16;  // square tiles, RT x RT per thread
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmDesc d = descs[tl.desc];
  const int m0 = tl.tm * BM, n0 = tl.tn * BN;
  int kbeg = 0, kend = d.k;
  if (d.flags & GEMM_B_UPPER) kend = min(kend, n0 + BN);  // op(B)[k][j] = 0 for k > j
  if (d.flags & GEMM_A_UPPER) kbeg = max(kbeg, m0);       // op(A)[i][k] = 0 for k < i
  const double *A = db + d.a;
  const double *B = db + d.b;
  double *C = db + d.c;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  double acc[RT][RT];
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < RT; ++c) acc[r][c] = 0.0;
  const int kstart = (kbeg / BK) * BK;
  int buf = 0;
  if (kstart < kend) load_tiles<BM>(A, B, d, m0, n0, kstart, kbeg, kend, As[0], Bs[0]);
  __syncthreads();
  for (int k0 = kstart; k0 < kend; k0 += BK) {
    if (k0 + BK < kend) load_tiles<BM>(A, B, d, m0, n0, k0 + BK, kbeg, kend, As[buf ^ 1], Bs[buf ^ 1]);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[RT], b[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) a[r] = As[buf][kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < RT; ++c) b[c] = Bs[buf][kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int gi = m0 + ty + 16 * r;
    if (gi >= d.m) continue;
#pragma unroll
    for (int c = 0; c < RT; ++c) {
      const int gj = n0 + tx + 16 * c;
      if (gj >= d.n) continue;
      double *cp = C + (long long)gi * d.ldc + gj;
      double v = d.alpha * acc[r][c];
      if (d.beta != 0.0) v = fma(d.beta, *cp, v);
      *cp = v;
    }
  }
}

// n <= 16 columns (right-hand sides): a block of 32 warps per 32 output rows,
// the n accumulators of a row in registers.  op(A) transposed: a thread per
// row and 32 k-lanes for one column (8 for several: their partial sums fill
// shared memory), coalesced along the rows; otherwise a warp per row.  Sums
// are reduced in a fixed order (deterministic).
constexpr int SKINNY_THREADS = 1024;
__global__ void __launch_bounds__(SKINNY_THREADS) gemm_skinny_kernel(const GemmDesc *__restrict__ descs,
                                                          const GemmTile *__restrict__ tiles,
                                                          double *__restrict__ db) {
  __shared__ double red[8][32][17];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmDesc d = descs[tl.desc];
  const double *A = db + d.a;
  const double *B = db + d.b;
  double *C = db + d.c;
  const int n = d.n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int m0 = tl.tm * 32;
  double acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0;
  if (d.ta && n == 1) {
    // one right-hand side: 32 k-lanes, four independent loads in flight per thread
    double (*red1)[33] = reinterpret_cast<double (*)[33]>(&red[0][0][0]);  // [32][33]
    const int i = m0 + tx;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (i < d.m) {
      const long long sb = d.tb ? 1 : d.ldb;  // stride of B's single column
      int k = ty;
      for (; k + 96 < d.k; k += 128) {
        const double x0 = A[(long long)k * d.lda + i], x1 = A[(long long)(k + 32) * d.lda + i];
        const double x2 = A[(long long)(k + 64) * d.lda + i], x3 = A[(long long)(k + 96) * d.lda + i];
        a0 = fma(x0, B[k * sb], a0);
        a1 = fma(x1, B[(k + 32) * sb], a1);
        a2 = fma(x2, B[(k + 64) * sb], a2);
        a3 = fma(x3, B[(k + 96) * sb], a3);
      }
      for (; k < d.k; k += 32) a0 = fma(A[(long long)k * d.lda + i], B[k * sb], a0);
    }
    red1[ty][tx] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (ty == 0 && i < d.m) {
      double sm = 0.0;
      for (int w = 0; w < 32; ++w) sm += red1[w][tx];
      double *cp = C + (long long)i * d.ldc;
      double v = d.alpha * sm;
      if (d.beta != 0.0) v = fma(d.beta, *cp, v);
      *cp = v;
    }
  } else if (d.ta) {
    const int i = m0 + tx;
    if (i < d.m && ty < 8)
      for (int k = ty; k < d.k; k += 8) {
        const double a = A[(long long)k * d.lda + i];
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < n) acc[c] = fma(a, d.tb ? B[(long long)c * d.ldb + k] : B[(long long)k * d.ldb + c], acc[c]);
      }
    if (ty < 8)
#pragma unroll
      for (int c = 0; c < 16; ++c) red[ty][tx][c] = acc[c];
    __syncthreads();
    if (ty == 0 && i < d.m) {
      for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][tx][c];
        double *cp = C + (long long)i * d.ldc + c;
        double v = d.alpha * s;
        if (d.beta != 0.0) v = fma(d.beta, *cp, v);
        *cp = v;
      }
    }
  } else if (n == 1) {
    // one right-hand side: a warp per row, four partial sums, one reduction
    const long long sb = d.tb ? 1 : d.ldb;
    for (int r = ty; r < 32; r += SKINNY_THREADS / 32) {
      const int i = m0 + r;
      if (i >= d.m) break;
      const double *arow = A + (long long)i * d.lda;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int k = tx;
      for (; k + 96 < d.k; k += 128) {
        a0 = fma(arow[k], B[k * sb], a0);
        a1 = fma(arow[k + 32], B[(k + 32) * sb], a1);
        a2 = fma(arow[k + 64], B[(k + 64) * sb], a2);
        a3 = fma(arow[k + 96], B[(k + 96) * sb], a3);
      }
      for (; k < d.k; k += 32) a0 = fma(arow[k], B[k * sb], a0);
      double sm = (a0 + a1) + (a2 + a3);
      for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
      if (tx == 0) {
        double *cp = C + (long long)i * d.ldc;
        double v = d.alpha * sm;
        if (d.beta != 0.0) v = fma(d.beta, *cp, v);
        *cp = v;
      }
    }
  } else {
    for (int r = ty; r < 32; r += SKINNY_THREADS / 32) {
      const int i = m0 + r;
      if (i >= d.m) break;
#pragma unroll
      for (int c = 0; c < 16; ++c) acc[c] = 0.0;
      const double *arow = A + (long long)i * d.lda;
      for (int k = tx; k < d.k; k += 32) {
        const double a = arow[k];
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < n) acc[c] = fma(a, d.tb ? B[(long long)c * d.ldb + k] : B[(long long)k * d.ldb + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < 16; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      if (tx == 0)
        for (int c = 0; c < n; ++c) {
          double *cp = C + (long long)i * d.ldc + c;
          double v = d.alpha * acc[c];
          if (d.beta != 0.0) v = fma(d.beta, *cp, v);
          *cp = v;
        }
    }
  }
}

}  // namespace

cudaError_t launch_gemm_phase(const Plan &p, const GemmPhase &ph, void *ws, cudaStream_t s) {
  if (ph.ntile == 0) return cudaSuccess;
  char *base = static_cast<char *>(ws);
  const GemmDesc *descs = reinterpret_cast<const GemmDesc *>(base + p.off_gdesc);
  const GemmTile *tiles = reinterpret_cast<const GemmTile *>(base + p.off_gtile) + ph.tile0;
  double *db = reinterpret_cast<double *>(base + p.off_dbl);
  if (ph.skinny)
    { gemm_skinny_kernel<<<ph.ntile, SKINNY_THREADS, 0, s>>>(descs, tiles, db); DDELM_COUNT_LAUNCH(); }
  else if (ph.tile == 16)
    { gemm_f64_kernel<16><<<ph.ntile, NT, 0, s>>>(descs, tiles, db); DDELM_COUNT_LAUNCH(); }
  else if (ph.tile == 64)
    { gemm_f64_kernel<64><<<ph.ntile, NT, 0, s>>>(descs, tiles, db); DDELM_COUNT_LAUNCH(); }
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Same kernels on caller-built tables (used by the static-scratch entry point).
cudaError_t launch_gemm_table(const GemmDesc *descs, const GemmTile *tiles, int ntiles, double *db, int skinny,
                              cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (skinny)
    { gemm_skinny_kernel<<<ntiles, SKINNY_THREADS, 0, s>>>(descs, tiles, db); DDELM_COUNT_LAUNCH(); }
  else
    { gemm_f64_kernel<64><<<ntiles, NT, 0, s>>>(descs, tiles, db); DDELM_COUNT_LAUNCH(); }
  return cudaGetLastError();
}

}  // namespace ddelm
