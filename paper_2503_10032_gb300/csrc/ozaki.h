// Tables of the tensor-core (BF16 slice) emulation of FP64 GEMMs.
#pragma once

#include <cuda_runtime.h>

namespace ddelm {

struct Plan;

// One operand seen as an R x K matrix with K the contraction index:
// element (r, k) = trans ? X[k*ld + r] : X[r*ld + k].  Its S slices are written
// as [S][Rpad][Kpad] BF16 (K contiguous, zero padded) and its row scales as R
// powers of two.
struct SliceDesc {
  long long x;      // dbase offset of the FP64 source
  long long out;    // element offset of the slices in the slice region
  long long scale;  // dbase offset of the R row scales
  int ld, trans;
  int R, K, Rpad, Kpad;
  int S, pad;
};

// C = alpha * op(A) op(B) + beta * C, m x n, with op(A) = slices sa (rows i) and
// op(B)^T = slices sb (rows j)
struct OzDesc {
  long long c, scaleA, scaleB;
  int m, n, ldc;
  int S, kc, Kpad;
  int RpadA, RpadB;
  int tmapA, tmapB;
  double alpha, beta;
};

// one 128 x bn output tile; only the 64-wide k blocks [kb0, kb1) can be
// nonzero in op(A)[tile rows] op(B)[:, tile columns] (triangular operands)
struct OzTile {
  int desc, tm, tn, kb0, kb1, pad0, pad1, pad2;
};

struct OzPhase {
  int slice0, nslice;    // SliceDesc range
  int desc0, ndesc;      // OzDesc range
  int tile0, ntile;      // OzTile range
  int max_rpad, max_kpad;
  int bn;                // tile width: 64 (four levels per group) or 128 (two)
  // the other tile width's tile list (ntile_alt = 0: none, the contraction is too
  // long for the four-level integer sums), for the autotuner
  int tile0_alt, ntile_alt, bn_alt;
  int overwrite;         // every product has beta = 0: the phase may run twice
  double flops, flops_alt;  // slice-pair flops of the two tile lists
  unsigned long long key;   // the phase's shape, the autotuner's cache key
};

cudaError_t launch_slices(const Plan &p, const OzPhase &ph, void *ws, cudaStream_t s);
cudaError_t launch_oz_gemm(const Plan &p, const OzPhase &ph, void *ws, cudaStream_t s);
cudaError_t preload_oz_kernels();

// the tile width the autotuner chose earlier in this process for a phase of
// this shape (0: none yet); defined with the autotuner
int tuned_tile_width(unsigned long long key);

}  // namespace ddelm
