// Internal declarations of libddelm: the device-side tables the host plan
// builds and the kernel launchers.  Every offset below is an element index
// into the double region of the caller's workspace (dbase) or into the int
// region (ibase); tables are position independent, so a plan is built once on
// the host and uploaded with one copy.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ddelm.h"
#include "ozaki.h"

namespace ddelm {

// every kernel launch of the library (the profiler attributes them to classes)
extern std::atomic<long long> g_kernel_launches;
#define DDELM_COUNT_LAUNCH() ::ddelm::g_kernel_launches.fetch_add(1, std::memory_order_relaxed)
// keeps the message ddelm_last_error() returns (per host thread)
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);
// keeps "problem rejected: <why>" for ddelm_last_error() (per host thread)
void record_plan_error(const std::string &why);

// ---------------------------------------------------------------- rows
// Rows of the local matrices other than the interior collocation rows.  They
// are written in two passes: the first evaluates tanh once per (point, neuron)
// and writes point values and fluxes; the second forms the rows that are
// combinations of rows of the first (the change of variables of Sec. 3.2 and
// the A_m corner rows), reading them instead of evaluating tanh again.
enum RowKind : int {
  ROW_POINT = 0,  // C phi = B phi = phi(x)
  ROW_DELTA = 1,  // Delta point: phi(x) to out0/out1 and F phi = (w . n)(1 - tanh^2) to out2/out3;
                  // second pass: phi(x) - alpha phi(x_a) - beta phi(x_b) ((T^i)^{-1} C phi)
  ROW_AM = 3,     // A_m corner row: mean edge fluxes (Sec. 3.2), second pass only
};

struct SpecialRow {
  int kind, sub;
  int comp, pad_;        // 0: phi and d phi/dn; 1 (biharmonic): (Lap phi and d Lap phi/dn) w_c1
  long long out0, out1;  // row starts in dbase (out1 < 0: single output)
  long long out2, out3;  // ROW_DELTA: K-bar Delta row and A_m Delta row (flux)
  long long ca, cb;      // rows holding phi(x_a), phi(x_b) (ROW_DELTA; < 0: none) or phi(corner) (ROW_AM)
  double x, y, nx, ny;
  double alpha, beta;
  // ROW_AM: per edge meeting the corner, its outward normal, the first of its
  // e flux rows (consecutive A_m rows) and e
  double am_n[2][2];
  long long am_f[2];
  int am_e[2];
};

// Interior collocation rows of subdomain `sub` go to rows [0, nI) of both
// K_c^i and K-bar^i; the point data come from the problem arrays.
struct SubDev {
  int M, nI, nB, nPi, nDl, nG, m, nE;
  long long w_off;    // first neuron of this subdomain in the packed w/b arrays
  long long int_off;  // first interior point
  long long eval_off; // first evaluation point
  // setup buffers (dbase offsets)
  long long oX;       // persistent [m x M]: the final Q of K_c^i after setup
  long long oK;       // where the feature kernels write K_c^i (oX or oY1: the
                      // Q updates alternate between the two so the last lands in oX)
  long long oKb;      // K-bar^i [m x M] (setup scratch)
  long long oY1, oY1b;  // the other Q buffers of K and K-bar [m x M] (setup scratch)
  long long oA;       // A_m^i [nG x M]
  long long oAbar;    // A-bar^i [nDl x M]
  long long oEval;    // phi at the evaluation points [nE x M]
  // persistent operators
  long long oV, oVb;       // R^{-1} of K and K-bar [M x M]
  long long oV3;           // third-pass R3^{-1} of K [M x M]
  long long oQG;           // Gamma rows of the final Q of K [nG x M]
  long long oKpE;          // K^+ E_Gamma [M x nG]
  long long oLam, oLamT;   // Lambda^i and its transpose [nG x nG]
  long long oPsi;          // Psi^i [nG x nG]
  long long oPhi, oPhiT;   // Phi^i and its transpose [nDl x nDl]
  long long oLam32, oLamT32, oPsi32, oPhi32, oPhiT32;  // MIXED: FP32 copies (float offsets)
  // solve-time vectors ([rows x R])
  long long oF;     // [nI + nB] x R data rows
  long long oT, oQtf, oY, oAy, oP;  // M x R, M x R, M x R, nG x R, nG x R
  long long oC;     // coefficients M x R
  long long oU;     // network values at the evaluation points nE x R
  int gpi_off, gdl_off, bnd_off;  // ibase offsets of R_Pi, R_Delta, boundary index maps
  int loc_off;      // first row of this subdomain in the local vector buffers (nG rows)
  long long dshift; // scale-gradient tables only: derivative block = value block + dshift
};

struct GemmDesc {
  long long a, b, c;  // dbase offsets
  int m, n, k;
  int lda, ldb, ldc;
  int ta, tb;  // 1: operand stored transposed
  int flags;   // GEMM_B_UPPER / GEMM_A_UPPER
  int syrk;    // 1: only the upper tiles of C are needed (C symmetric)
  double alpha, beta;
};
enum { GEMM_B_UPPER = 1, GEMM_A_UPPER = 2 };

struct GemmTile {
  int desc, tm, tn, pad;
};

struct CholDesc {
  long long g;  // in: symmetric matrix (upper triangle read); FP64 passes factor it in place
  long long v;  // out: R^{-1} (upper, full square written)
  long long z;  // out: sqrt(eps2) R^{-1} (ridge passes); < 0 for none
  long long w;  // FP32 passes: work buffer of 2 M^2 floats
  int M, m;     // order, rows of the matrix whose Gram g is (for the shift)
  int ridge;    // 1: add eps^2 = eps_rel^2 tr(G)/M (the ridge of the local problem)
  int shift_kind;  // 0 none, 1 shift_rel * tr(G + eps^2 I), 2 shift_rel * max diag(G + eps^2 I)
  int prec;     // 0 FP64, 1 FP32, 2 double-FP32
  int band;     // > 0: G and R vanish beyond this many superdiagonals
  int status;   // index into the status array
  int inv_block; // > 0: only the inv_block x inv_block diagonal blocks of R^{-1} (the rest by GEMMs)
  int ld;       // leading dimension of g and v (0: M); a diagonal block of a larger matrix
  int mode;     // 0 factor (and invert); 1 blocked factorisation's first step: add the ridge and
                // shift to the diagonal of the whole matrix, write eps, zero v (M x M, leading dim M)
  double eps_rel;
  double shift_rel;
  long long epsout;  // >= 0: dbase offset receiving eps = sqrt(eps^2) (the ridge block is formed later)
};

struct MatopDesc {
  long long a, b, c;
  int M, op;   // op 0: C = -I ; op 1: C = I - A/2 + 3/8 B - 5/16 D ; op 2: lower(C) = upper(C)^T ;
               // op 3: C = A ; op 4: C = A - I ; op 5: C = b A (b: the scalar at offset b)
  int status;  // op 1: set when max |A| exceeds the range of the series
  long long d; // op 1: third-order term (< 0: none)
};

// FP64 -> FP32 copy of n elements (dbase offset src, FP32-region offset dst)
struct ConvSeg {
  long long src, dst, n;
};

struct MatopPhase {
  int desc0, ndesc;
};

// one step of the setup sequence
enum StepKind : int { STEP_GEMM = 0, STEP_CHOL = 1, STEP_MATOP = 2, STEP_FEAT = 3 };
struct Step {
  int kind, idx;
};

// ---------------------------------------------------------------- scale gradient
// dL/ds for the hidden-layer scale s (w = s w_hat, b = s b_hat, Sec. 2.2) by
// reverse mode at the solution: the persistent kernel forms, from the adjoint
// solution b-bar = S_theta^{-1} mu-bar, the cotangent vectors of every local
// operator application (a "bank" of interface vectors); per subdomain these
// become low-rank cotangents of K_c, K-bar, A_m, A-bar and the evaluation
// matrix (through d(K^+) for the ridge pseudo-inverse), which are contracted
// with the matrices' analytic s-derivatives.
enum ScaleDl { SD_BB = 0, SD_NEGBB, SD_MU, SD_VR, SD_PVR, SD_WR, SD_WRS, SD_PVSR, SD_VSR, SD_WB, SD_PVB, SD_VB, N_SD };
enum ScalePi {
  SP_DPI = 0, SP_PPI, SP_MPF, SP_GF, SP_RNUR, SP_NUR, SP_DNUR,             // right-hand-side program
  SP_PIA, SP_PIC, SP_PID, SP_RNURS, SP_RAS, SP_PSIS, SP_DPIPSI, SP_RAPPI,  // combinations with S_theta mu
  SP_PSI2, SP_S2, SP_MPIF,                                                 // reconstruction
  SP_MPIFB, SP_S2B, SP_PSI2B, SP_GFB, SP_NUB, SP_DNUB, SP_RNUB, SP_ZLV,    // reverse pass
  SP_MPFB, SP_MPIBS, SP_RABS, SP_PSIBS, SP_PPIB, SP_DPIB, SP_PIB, SP_PIE, SP_ZERO, N_SP
};
// per subdomain: the re-assembled local matrices (value block; their
// s-derivatives at + dshift) and the factored cotangents and products
struct ScaleSub {
  long long Ks, Kbs, As, Abs, Es, dshift;
  long long Bc, LA, LG, Ac, RAG, ybar, VtA, RK, QGB, LK, T2, Rt, Vty, PF, WFm;
  long long t1, t2, t3, t4, RKb, LKb, V3QGB, V3VtA, V3Vty, V3Rt;
  long long OK, OG, OA, OKb, OAb, OE;
};
// one block dot product sum_{r<rows, c<cols} a[r lda + c] b[r ldb + c] of subdomain sub
struct DotDesc {
  long long a, b;
  int rows, cols, lda, ldb;
  int sub, role;
  double coef;
};
enum { DOT_LIN = 0, DOT_E2K = 1, DOT_KDK = 2, DOT_E2KB = 3, DOT_KBDKB = 4 };

// ---------------------------------------------------------------- plan
struct GemmPhase {
  int desc0, ndesc;  // into the descriptor table
  int tile0, ntile;  // into the tile table
  int skinny;        // 1: every n <= 16; tiles are 32-row blocks (tn = 0)
  int tile = 64;     // otherwise the edge of the square output tiles: 64, or 16 for tiny products
};

struct CholPhase {
  int desc0, ndesc;
};

struct Plan {
  ddelm_sizes sz{};
  int n_sub = 0, n_rhs = 1, op = 0;
  int max_M = 0;
  // host copies of the tables
  std::vector<SubDev> subs;
  std::vector<SpecialRow> rows;
  std::vector<GemmDesc> gdesc;
  std::vector<GemmTile> gtile;
  std::vector<CholDesc> cdesc;
  std::vector<int> ints;  // gpi, gdl, bnd maps, owner maps, task lists
  // phases (indices into the tables)
  std::vector<GemmPhase> setup_gemm;  // filled in order; see api.cu for the sequence
  std::vector<double> gemm_flops;      // algorithmic flops per descriptor
  std::vector<double> phase_flops;     // per GEMM phase
  double chol_flops = 0.0;             // all Cholesky + inverse passes of one setup
  // named ranges into ints
  int o_pi_own = 0;   // per Pi point: 4 x (sub, local) pairs, -1 padded
  int o_dl_own = 0;   // per Delta point: 4 x (sub, local), -1 past its owners (2, or 4 for the
                      // cross points of vanilla DDELM)
  int o_tasks_pi = 0, n_tasks_pi = 0;  // (sub, local Pi row)
  int o_tasks_dl = 0, n_tasks_dl = 0;  // (sub, local Delta row)
  int o_tasks_g = 0, n_tasks_g = 0;    // (sub, local Gamma row)
  int o_tasks_c = 0, n_tasks_c = 0;    // (sub, coefficient row j < M)
  int o_dl_rows = 0;                    // per Delta point: its owners' slab rows (4, -1 past the owners)
  int o_gam_rows = 0;                   // per local interface row: those rows of its Delta point (-1 on Pi)
  int o_bnd_map = 0;                    // local boundary -> global Dirichlet index
  int o_bnd_own = 0;                    // per global Dirichlet point: 2 x (sub, local row)
  // workspace layout
  size_t bytes_tables = 0, bytes_total = 0;
  size_t off_subs = 0, off_rows = 0, off_gdesc = 0, off_gtile = 0, off_cdesc = 0, off_ints = 0;
  size_t off_dbl = 0;      // byte offset of the double region
  long long n_dbl = 0;     // doubles in the region
  long long o_w = 0, o_b = 0, o_xint = 0, o_aint = 0, o_gaint = 0;  // problem data
  long long o_fc = 0;    // per neuron (2 w_x, 2 w_y, 2 b, 2 |w|^2)
  long long o_exp2 = 0;  // 2^(-j/256), j < 256 (the feature tanh)
  long long o_status = 0;  // int status slots (in ints region? kept as doubles)
  long long o_eps = 0;     // per local matrix: eps of the ridge (2 per subdomain)
  long long o_fin = 0, o_gin = 0, o_cout = 0, o_muout = 0, o_uout = 0;  // solve staging
  // MIXED: FP32 region (dbase offset o_f32, n_f32 floats): operator copies and
  // the inner CG's Delta vectors (6), Pi vectors (7) and local slabs (8)
  long long o_f32 = -1, n_f32 = 0;
  long long f_Sinv = 0, f_C1 = 0, f_C2 = 0, f_C3 = 0, f_dl = 0, f_pv = 0, f_slab = 0;
  std::vector<ConvSeg> conv;
  size_t off_conv = 0;
  // coarse
  int n_pi = 0, n_dl = 0;
  long long o_Dpp = 0, o_Spi = 0, o_Vpi = 0, o_Sinv = 0, o_C1 = 0, o_C2 = 0, o_C3 = 0, o_SpiR = 0;
  // CG vectors / scratch
  long long o_cg = 0, n_cg = 0;
  long long o_loc = 0;  // local vector buffers: several [sum nG x R] slabs
  int sum_nG = 0;
  // inspection copies
  long long o_keepX = -1;
  bool keep = false;
  ddelm_options opt{};
  // setup waves: subdomains [w*wave, (w+1)*wave) share the scratch slots
  int wave = 1, n_waves = 1;
  // phase layout in setup_gemm: wave w phase q (0..10) at 11*w + q, then the
  // coarse (4), solve (5) and adjoint (6) phases from these offsets
  int ph_coarse = 0, ph_solve = 0, ph_adj = 0;
  // chol phases (referenced by the step list), coarse chol
  std::vector<CholPhase> chol_passes;
  CholPhase chol_coarse{};
  std::vector<MatopDesc> mdesc;
  std::vector<MatopPhase> matop_phases;
  std::vector<Step> steps;  // the per-subdomain part of the setup, in order
  std::vector<int> setup_levels;  // per setup GEMM phase: BF16 slice levels (MIXED)
  std::vector<int> wave_row0;     // special rows of wave w: [wave_row0[w], wave_row0[w+1]); then evaluation rows
  int scheme = DDELM_SCHEME_FP64CQR3;
  int n_pass = 2;        // Cholesky passes before the last one
  bool polish = false;   // last factor corrected by the series (I + E)^{-1/2}
  bool tri_v = true;     // V and the last factor are upper triangular
  double chol_flops32 = 0.0;  // the part of chol_flops done in FP32
  size_t off_mdesc = 0;
  // tensor-core emulation of the setup GEMMs (precision MIXED)
  bool mixed = false;
  int tc_tiles = 0;               // tensor-core tile shapes allowed (the tc_tiles option)
  bool autotune = false;          // the autotuner's alternative lists are planned
  int tune_from_cache = 0;        // phases whose width an earlier handle's autotuner chose
  bool maps_grp = false, maps_al = false;  // tensor-map families some tile list uses
  std::vector<SliceDesc> sdesc;
  std::vector<OzDesc> odesc;
  std::vector<OzTile> otile;
  std::vector<OzPhase> oz_phase;  // parallel to setup_gemm; ntile == 0: FP64 engine
  size_t off_sdesc = 0, off_odesc = 0, off_otile = 0, off_tmaps = 0, off_slices = 0;
  size_t bytes_slices = 0;
  double oz_flops = 0.0;          // BF16 tensor flops of one setup
  double slice_bytes = 0.0;       // HBM bytes of the slicing kernels of one setup
  // scale gradient (ddelm_backward with a scale output)
  double inv_scale = 0.0;                 // 1 / s
  // row weights of the biharmonic system (every derivative of order k times H^k,
  // H the subdomain size): interior rows (and f) times w_int = H^4, the second
  // component's point rows (and its boundary data) times w_c1 = H^2, flux rows
  // times w_f0 = H (first component) and w_f1 = H^3 (second); 1 for the other
  // operators
  double w_int = 1.0, w_c1 = 1.0, w_f0 = 1.0, w_f1 = 1.0;
  // automatic double-FP32 first factors: the Cholesky descriptors that take
  // them and their FP64 shifts, for the fallback to FP64 factors when such a
  // setup fails (a hard problem where the first factor's accuracy is marginal)
  bool dw_auto = false;
  std::vector<std::pair<int, double>> dw_fallback;
  int nb0 = 0;                            // Dirichlet points of the first component
  std::vector<long long> slot_begin, slot_end;  // contiguous setup-scratch extent of each wave slot
  std::vector<SubDev> ssubs;              // feature tables writing into the scale buffers
  std::vector<SpecialRow> srows;
  std::vector<int> wave_erow0;            // evaluation rows of wave w in srows: [wave_erow0[w], wave_erow0[w+1])
  std::vector<ScaleSub> scsub;
  std::vector<DotDesc> dots;
  std::vector<int> wave_dot0;             // dot descriptors of wave w
  std::vector<GemmPhase> sc_coarse;       // coarse chain of the cotangents
  std::vector<std::vector<GemmPhase>> sc_wave;  // per wave: the products of the factored cotangents
  int sc_JL = 0, sc_JP = 0, sc_JF = 0, sc_Jc = 0, sc_NK = 0, sc_NAG = 0;
  long long o_bank_dl = 0, o_bank_pi = 0;  // N_SD Delta vectors, N_SP Pi vectors ([n x R] each)
  long long o_cSb = 0, o_cC1b = 0, o_cC2b = 0, o_cC3b = 0, o_cDb = 0, o_cDX = 0, o_cT1 = 0, o_cT3 = 0, o_cSPb = 0;
  long long o_gs = 0;                       // per dot descriptor, then per subdomain, then the total
  size_t off_ssubs = 0, off_srows = 0, off_scsub = 0, off_dots = 0;
  std::string err;
};

int build_plan(const ddelm_problem *prob, Plan &plan);
int build_mixed(Plan &plan, long long &dbl_cursor);
int build_scale(Plan &plan, long long &dbl_cursor);
int encode_tensor_maps(const Plan &plan, void *ws, std::vector<unsigned char> &maps);

// ---------------------------------------------------------------- launchers
cudaError_t launch_features(const Plan &p, void *ws, int wave, cudaStream_t s);
cudaError_t launch_gemm_phase(const Plan &p, const GemmPhase &ph, void *ws, cudaStream_t s);
cudaError_t launch_chol_phase(const Plan &p, const CholPhase &ph, void *ws, cudaStream_t s);
cudaError_t launch_matop_phase(const Plan &p, const MatopPhase &ph, void *ws, cudaStream_t s);
cudaError_t launch_convert_f32(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_coarse_assembly(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_fill_identity(double *dst, int n, double diag, cudaStream_t s);
cudaError_t launch_gather_rhs(const Plan &p, void *ws, const double *f_int, const double *g_bnd,
                              cudaStream_t s);
cudaError_t launch_adjoint_init(const Plan &p, void *ws, const double *grad_c, const double *grad_u, cudaStream_t s);
cudaError_t launch_copy_c_to_y(const Plan &p, void *ws, cudaStream_t s);
cudaError_t launch_adjoint_scatter(const Plan &p, void *ws, double *grad_f, double *grad_g, cudaStream_t s);
cudaError_t launch_gemm_table(const GemmDesc *descs, const GemmTile *tiles, int ntiles, double *db, int skinny,
                              cudaStream_t s);
cudaError_t launch_chol_table(const CholDesc *descs, int n, int maxM, double *db, int *status, cudaStream_t s);
struct CgArgs {
  double *mu_out;   // [n_pi + n_dl] x R or null
  double *c_out;    // [sum M] x R or null
  int max_iters;
  double tol;
  double theta;
  int mode = 0;  // 0 solve, 1 adjoint, 2 residual at a given mu, 3 solve for a given right-hand side,
                 // 4 the scale-gradient vectors (after mode 1)
  int max_refine = 8;  // MIXED: outer refinement sweeps
};
cudaError_t launch_cg(const Plan &p, void *ws, const CgArgs &a, cudaStream_t s);
// scale gradient launchers (features of wave w and their s-derivatives into the
// scale buffers; the per-subdomain operands; the block dot products; the total)
cudaError_t launch_scale_features(const Plan &p, void *ws, int wave, cudaStream_t s);
cudaError_t launch_scale_gather(const Plan &p, void *ws, int wave, double theta, cudaStream_t s);
cudaError_t launch_scale_dots(const Plan &p, void *ws, int wave, cudaStream_t s);
cudaError_t launch_scale_total(const Plan &p, void *ws, double eps_rel, cudaStream_t s);
void cg_vectors(const Plan &p, void *ws, double **mu, double **rhs, double **res);

}  // namespace ddelm
