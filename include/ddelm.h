/*
 * ddelm.h -- C ABI of the GB300 DDELM-NN library (libddelm.so).
 *
 * The library solves the coarse-space, Neumann-Neumann accelerated domain
 * decomposition of extreme learning machines of arXiv 2503.10032 for 2-D
 * second-order problems on a rectangle split into nx x ny subdomains:
 *
 *   setup  (ddelm_setup):  assembly of the local ELM collocation matrices
 *          K_c^i (Sec. 2.2.1 with the change of variables of Sec. 3.2),
 *          the Neumann matrices K-bar^i (Sec. 3.1), the modified flux rows
 *          A_m^i (Sec. 3.2); factorisation of every local least-squares
 *          problem; the local operators from which D_ab = -A_a K^+ B_b
 *          (Sec. 3), K K^+ and P = A-bar K-bar^+ B-bar (Sec. 3.1) are
 *          applied; the coarse matrix S_Pi assembled in full and factored
 *          (Sec. 3).
 *   solve  (ddelm_solve): for given forcing / boundary data, the right-hand
 *          side of Eq. (nn-mixed), CG on Eq. (nn-mixed) for mu_Delta, then
 *          [c; mu_Pi] = K~^+ (f~ - B~ mu_Delta), Eq. (coarse_sol_2), and the
 *          network values at caller-given points.
 *   backward (ddelm_backward): the adjoint of solve with respect to the
 *          right-hand-side values and the hidden-layer scale (gradients of a
 *          loss given dL/dc or dL/du).
 *
 * Conventions shared by every entry point:
 *   - All floating-point data are IEEE double.  Host pointers are read during
 *     the call only; device pointers are owned by the caller and must stay
 *     valid until the stream work of the call has completed.
 *   - Subdomain (ix, iy) has index iy*nx + ix and covers
 *     [x0 + ix*hx, x0 + (ix+1)*hx] x [y0 + iy*hy, y0 + (iy+1)*hy].
 *   - Grid edges: horizontal edge (ix, vy) has id vy*nx + ix; vertical edge
 *     (vx, iy) has id nx*(ny+1) + vx*ny + iy.  An edge with e points carries
 *     them at start + k/(e+1) * (end - start), k = 1..e, start = the vertex
 *     with the smaller coordinate.
 *   - Dirichlet data g are given on the global boundary list: the points of
 *     every edge on the outer boundary in edge-id order, then every grid
 *     vertex on the outer boundary in order vy*(nx+1) + vx.
 *   - Interface unknowns: Gamma = Pi (interior grid vertices, order
 *     (vy-1)*(nx-1) + (vx-1)) followed by Delta (points of the interior edges,
 *     edge-id order, k = 1..e).  With the change of variables on, mu_Pi are
 *     the coefficients of the edge-linear coarse functions of Sec. 3.2 and
 *     mu_Delta the remaining values (mu = T mu' of Sec. 3.2).
 *   - Arrays with a right-hand-side dimension are row-major [rows x n_rhs].
 *   - Return value: DDELM_OK or a negative status; no call aborts, traps or
 *     exits.  After a CUDA error the handle must be destroyed.
 *
 * Numerical readings fixed by this library (the paper is silent on them):
 *   - K^+ is the pseudo-inverse of K augmented by rows eps*I with zero data
 *     (a ridge term eps^2 |c|^2 in every local least-squares loss), with
 *     eps^2 = eps_rel^2 * |K|_F^2 / M, separately for K^i and K-bar^i;
 *     eps_rel = 0 gives the Moore-Penrose pseudo-inverse.
 *   - F phi = (w . n)(1 - tanh^2(w.x + b)), n the subdomain's outward normal.
 *   - A-bar^i uses the Delta rows of K_c^i (the (T^i)^{-1} C phi rows).
 *   - The corner row of A_m^i sums, over the two edges of subdomain i that
 *     meet the corner, the mean flux over the corner and the edge's e points.
 */
#ifndef DDELM_H
#define DDELM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDELM_OK 0
#define DDELM_ERR_INVALID_ARG (-1)    /* bad sizes, null pointers, workspace too small */
#define DDELM_ERR_RANK_DEFICIENT (-2) /* a local factorisation failed: a Cholesky pivot was not positive, or a series scheme met max |E| > 1e-4 (info: subdomain) */
#define DDELM_ERR_NOT_CONVERGED (-3)  /* CG reached max_iters, or the data / a CG scalar is not finite
                                         (NaN or Inf); outputs are still written */
#define DDELM_ERR_CUDA (-4)           /* a CUDA runtime call failed */
#define DDELM_ERR_TIMEOUT (-5)        /* a device-side grid barrier gave up waiting */
#define DDELM_ERR_UNSUPPORTED (-6)    /* an option or size this build does not support */

#define DDELM_OP_POISSON 0    /* L = -Laplacian */
#define DDELM_OP_DIFFUSION 1  /* L = -div(a grad), a and grad a given at x_int */
#define DDELM_OP_BIHARMONIC 2 /* L = Laplacian^2, the coupled system of Sec. 2.1: u and Lap u given on
                                 the boundary; u and Lap u continuous across the interface and both
                                 normal derivatives balanced, so every boundary and interface point
                                 carries two unknowns (component 0: u, component 1: Lap u). The
                                 Dirichlet list and the interface are numbered component 0 first:
                                 g = [u on the n_bnd/2 points; Lap u on the same points],
                                 Gamma = [Pi u; Pi Lap u; Delta u; Delta Lap u]. The change of
                                 variables and A_m (Sec. 3.2) act on each component separately.
                                 The loss terms are reweighted: every derivative of order k times
                                 H^k, H = sqrt(hx hy) the subdomain size (interior rows and f
                                 times H^4, the second component's point rows and boundary data
                                 times H^2, flux rows times H and H^3); mu of the second
                                 component is v = H^2 Lap u. */

#define DDELM_PREC_FP64 0  /* every step in FP64 */
#define DDELM_PREC_MIXED 1 /* FP32 inner CG with FP64 true-residual refinement */

/* Factorisation schemes of the ridge problems [K; eps I] (Sec. 2.2 pseudo-inverses):
 *  FP64CQR3: shifted CholeskyQR3, every Cholesky factor in FP64 (the FP64 path);
 *  FP32:     shifted CholeskyQR with FP32 Cholesky factors used only as
 *            preconditioners (every update of Q, the ridge block and R^{-1} stays
 *            FP64-exact), then one unshifted FP32 pass whose residual
 *            E = V^T G V - I is removed by V (I - E/2 + 3/8 E^2 - 5/16 E^3).
 *  CQR2_SERIES: two FP64 Cholesky passes (the first shifted); the third
 *            Gram G is within ~1e-5 of I and (I + E)^{-1/2}, E = G - I, is
 *            taken from its series to third order instead of a Cholesky.
 * The series are checked: max |E| > 1e-4 fails the setup (RANK_DEFICIENT).
 * Automatic: FP64CQR3 in FP64 precision; in MIXED, FP32 once some subdomain has
 * M >= 512 (where the O(M^3) FP64 Cholesky of one SM per matrix dominates),
 * else CQR2_SERIES_DW (defined below), and ddelm_setup falls back to
 * CQR2_SERIES when that setup reports a failed factorisation. */
#define DDELM_SCHEME_AUTO 0
#define DDELM_SCHEME_FP64CQR3 1
#define DDELM_SCHEME_FP32 2
#define DDELM_SCHEME_CQR2_SERIES 3
/* CQR2_SERIES_DW: as CQR2_SERIES, the factor of the shifted first pass computed
 * in double-FP32 arithmetic (pairs of FP32 numbers, about 46 significant bits)
 * on the FP32 pipe instead of FP64: it is a preconditioner only (every product
 * with it is FP64-exact) and the pass's shift covers the 2^-46 rounding.  The
 * unshifted second pass stays FP64 (its factor sets the |E| the series must
 * remove). */
#define DDELM_SCHEME_CQR2_SERIES_DW 4

typedef struct ddelm_options {
  double theta;           /* Eq. (nn-mixed) mixing weight; the paper uses 0.999 */
  double eps_rel;         /* ridge of the local least-squares problems (see above) */
  double tol;             /* stop when the relative residual of Eq. (nn-mixed) < tol */
  int max_iters;          /* CG iteration cap (per refinement sweep in MIXED) */
  int use_change_of_vars; /* 1: K_c^i (Sec. 3.2); 0: plain C phi rows */
  int precision;          /* DDELM_PREC_FP64 or DDELM_PREC_MIXED */
  int max_refine;         /* MIXED: outer refinement sweeps */
  int keep_matrices;      /* 1: keep the assembled K_c^i, K-bar^i, A_m^i for ddelm_inspect */
  int setup_wave;         /* subdomains whose setup scratch coexists (0: as many as fit 48 GiB) */
  int setup_scheme;       /* factorisation of [K; eps I]: DDELM_SCHEME_* (0: automatic) */
  int setup_passes;       /* DDELM_SCHEME_FP32: shifted FP32 passes before the last (0: automatic) */
  int disable_graphs;     /* 1: issue every launch directly; 0: the setup (from the first
                             ddelm_refactor) and the solve (from a handle's second ddelm_solve)
                             are captured once as CUDA graphs and replayed */
  int barrier_timeout_ms; /* a grid barrier of the interface solve gives up (DDELM_ERR_TIMEOUT)
                             after waiting this long (0: 2000) */
  int inject_barrier_stall; /* tests only: every grid barrier of the interface solve waits for one
                             arrival more than the grid has, so it can end only by its time limit;
                             the kernel then returns and the call reports DDELM_ERR_TIMEOUT */
  int plain_flux_corners; /* 0: the modified flux A_m of Sec. 3.2 (corner rows = mean fluxes along
                             the two edges); 1: the plain flux rows A of Eq. (ddelm), the corner
                             row being the sum, over the two edges of the subdomain that meet the
                             corner, of the flux at the corner with that edge's normal */
  int vanilla;            /* 1: vanilla DDELM (Sec. 2.2.1, Eq. (schur)), no coarse space: Pi is empty
                             and every cross point is an interface unknown of its four subdomains,
                             numbered first in Delta (in the order (vy-1)(nx-1) + vx-1), with the
                             plain corner flux row above; requires theta = 0 (the NN map of
                             Sec. 3.1 belongs to the coarse-space method). 0: the coarse space
                             of Sec. 3 */
  int autotune;           /* MIXED: 1 = the first setup of a handle (ddelm_setup) times both tile
                             shapes of every tensor-core GEMM phase whose products overwrite their
                             output (128 x 64 tiles with four slice levels per group, 128 x 128
                             with two) and keeps the faster for every later setup; phases that
                             accumulate keep the fixed rule (128 wide when every contraction is
                             longer than 1024).  The choices are cached for the process by phase
                             shape, so later handles of the same problem reuse them without
                             timing.  Results are FP64-exact either way.  0: the rule */
  int trim_levels;        /* experiments only (MIXED): slice levels taken off the tensor-core
                             products of the classes in trim_mask (at least 3 remain), to measure
                             what each class's level count buys; 0 in normal use */
  int trim_mask;          /* 1 Grams after the first pass, 2 Q and ridge-block updates, 4 products
                             of triangular factors, 8 local operators and their inputs, 16 the
                             first Gram */
  int chol_blocked;       /* MIXED, experimental: 1 = the FP64 Cholesky passes of subdomains with
                             M > 128 are blocked (the FP64 kernel factors and inverts the 128-wide
                             diagonal blocks, tensor-core GEMMs form the panels and the trailing
                             updates); 0 (the default) = one CTA factors a whole matrix.  The
                             blocked panels multiply by the explicit inverse of the diagonal
                             block, which is not backward stable: with eps_rel = 1e-8 the second
                             pass's Gram (condition ~1e11) fails the series check; use it for
                             well-conditioned problems (eps_rel >= 1e-4, where it matches the
                             unblocked factor to 1e-12 and saves ~1.8 ms per setup at 8x8/M=400) */
  int tc_tiles;           /* MIXED tensor-core tile shapes: 0 = the all-levels shape (128 x 48
                             tiles, every slice level of a 32-wide k block in one shared-memory
                             stage) by rule, with the level-group shape (128 x 64 or 128 x 128,
                             see autotune) as the autotuner's alternative; 1 = the level-group
                             shapes only (the rule and the other width); 2 = the all-levels shape
                             only; 3 = the 128 x 64 level-group shape only (its exact integer
                             level combination, for every contraction length).  Contractions
                             longer than 16384 always take the 128-wide level-group shape.
                             FP64-exact either way */
} ddelm_options;

typedef struct ddelm_problem {
  int nx, ny;               /* subdomains per direction (>= 1 each) */
  double x0, x1, y0, y1;    /* the rectangle */
  int op;                   /* DDELM_OP_POISSON, DDELM_OP_DIFFUSION or DDELM_OP_BIHARMONIC */
  int n_rhs;                /* right-hand sides solved together (>= 1) */
  const int *M;             /* [n_sub] neurons per subdomain (1..1024) */
  const double *w_hat;      /* [sum M][2] hidden weights before scaling */
  const double *b_hat;      /* [sum M] hidden biases before scaling */
  double scale;             /* s: w = s*w_hat, b = s*b_hat */
  const int *n_int;         /* [n_sub] interior collocation points per subdomain */
  const double *x_int;      /* [sum n_int][2] interior points, subdomain by subdomain */
  const double *a_int;      /* [sum n_int] coefficient a (DIFFUSION only, else NULL) */
  const double *grad_a_int; /* [sum n_int][2] grad a (DIFFUSION only, else NULL) */
  const int *edge_pts;      /* [n_edges] points strictly inside every grid edge */
  const int *n_eval;        /* [n_sub] evaluation points per subdomain (NULL: none) */
  const double *x_eval;     /* [sum n_eval][2] evaluation points */
  ddelm_options opt;
} ddelm_problem;

typedef struct ddelm_sizes {
  int n_sub, n_edges;
  int n_bnd;           /* length of the global Dirichlet list (biharmonic: both components) */
  int n_pi, n_delta;   /* |Pi|, |Delta| (biharmonic: both components) */
  long long sum_M, sum_int, sum_eval;
  size_t workspace_bytes; /* device workspace ddelm_setup needs */
  size_t upload_bytes;    /* host-to-device bytes ddelm_setup copies (tables + problem data) */
} ddelm_sizes;

typedef struct ddelm_solve_info {
  int iterations;        /* CG iterations (all sweeps) */
  int refinements;       /* MIXED: outer sweeps taken */
  double rel_residual;   /* max over right-hand sides of the true FP64
                            |b_theta - S_theta mu| / |b_theta| at exit */
  double ms_total;       /* device time of the call (stream events) */
} ddelm_solve_info;

typedef struct ddelm_handle ddelm_handle;

/* Sizes derived from the problem (host only, no GPU work).
 * Returns DDELM_ERR_INVALID_ARG on inconsistent input. */
int ddelm_query(const ddelm_problem *prob, ddelm_sizes *out);

/* Builds the handle and runs the whole setup on `stream` (a cudaStream_t;
 * NULL = default stream): uploads the problem, assembles the local matrices,
 * factorises them, forms the local and coarse operators.  d_workspace is a
 * device buffer of at least ddelm_sizes.workspace_bytes bytes (256-byte
 * aligned), owned by the caller and used by the handle until ddelm_destroy.
 * The call returns after the setup work has completed on the stream.
 * info_sub (nullable) receives the first rank-deficient subdomain. */
int ddelm_setup(const ddelm_problem *prob, void *d_workspace, size_t workspace_bytes,
                void *stream, ddelm_handle **out, int *info_sub);

/* Re-runs the whole setup (assembly, factorisation, local and coarse
 * operators) from the problem data already resident in the workspace, on
 * `stream`, without host work or host-device copies; the call returns after
 * the work has completed.  Status as ddelm_setup. */
int ddelm_refactor(ddelm_handle *h, void *stream, int *info_sub);

/* One solve for new data.  Device inputs: d_f_int [sum n_int][n_rhs] forcing
 * at the interior points, d_g_bnd [n_bnd][n_rhs] Dirichlet data.  Device
 * outputs (nullable): d_c [sum M][n_rhs] network coefficients,
 * d_mu [n_pi + n_delta][n_rhs] interface unknowns (Pi first),
 * d_u_eval [sum n_eval][n_rhs] network values at the evaluation points.
 * info (host, nullable) is filled after the stream work completed. */
int ddelm_solve(ddelm_handle *h, const double *d_f_int, const double *d_g_bnd, double *d_c,
                double *d_mu, double *d_u_eval, ddelm_solve_info *info, void *stream);

/* Adjoint of the solve: the map (f, g) -> c of ddelm_solve is linear, and this
 * call applies its exact transpose.  Given device cotangents d_grad_c
 * [sum M][n_rhs] (dL/dc, nullable) and d_grad_u [sum n_eval][n_rhs] (dL/du at
 * the evaluation points, nullable, u = Phi_eval c), writes d_grad_f
 * [sum n_int][n_rhs] = dL/df and d_grad_g [n_bnd][n_rhs] = dL/dg (device,
 * nullable).  Reuses the setup's factors: the transposed local products with
 * V, R3^{-1}, Q_Gamma, A_m and K^+ E_Gamma, the transposed coarse steps, and
 * one CG on the symmetric S_theta.
 *
 * h_grad_scale (host, nullable) receives dL/ds for the hidden-layer scale s
 * (w = s w_hat, b = s b_hat, Sec. 2.2): the derivative of the loss through c and
 * u at the data and solution of the handle's most recent ddelm_solve (a
 * ddelm_interface_residual or ddelm_refactor call after it makes the call
 * return DDELM_ERR_INVALID_ARG, as does scale = 0).  It is computed in reverse
 * mode at that solution with the same adjoint solve and the setup's factors (no
 * further setup or solve): every application of a local operator (Lambda^i,
 * Psi^i, Phi^i, K^+ E_Gamma, the coarse matrices) and of K^+ to the data
 * contributes its output cotangent times its input; these become, through the
 * derivative of the ridge pseudo-inverse, low-rank cotangents of K_c^i, K-bar^i,
 * A_m^i, A-bar^i and the evaluation matrix, contracted with their analytic
 * s-derivatives (the ridge eps^2 = eps_rel^2 |K|_F^2 / M included).  It uses
 * the setup scratch of the workspace.  Not available for DDELM_OP_BIHARMONIC
 * (DDELM_ERR_UNSUPPORTED when h_grad_scale is given).
 *
 * info as in ddelm_solve (iterations of the adjoint CG; rel_residual is not
 * computed and reads 0). */
int ddelm_backward(ddelm_handle *h, const double *d_grad_c, const double *d_grad_u, double *d_grad_f,
                   double *d_grad_g, double *h_grad_scale, ddelm_solve_info *info, void *stream);

/* The interface residual of Eq. (nn-mixed) at a given mu: with the handle's
 * factors and the data (f, g) (device, as in ddelm_solve), writes
 * d_r [n_delta][n_rhs] = b_theta - S_theta mu_Delta for the caller's
 * d_mu_delta [n_delta][n_rhs], and (nullable) the coefficients d_c
 * [sum M][n_rhs] and d_u_eval of Eq. (coarse_sol_2) at that mu (all device).
 * With f = g = 0 it applies -S_theta and the linear part of the
 * reconstruction.  Synchronous; DDELM_ERR_TIMEOUT on a barrier timeout. */
int ddelm_interface_residual(ddelm_handle *h, const double *d_f_int, const double *d_g_bnd,
                             const double *d_mu_delta, double *d_r, double *d_c, double *d_u_eval, void *stream);

/* Solves S_theta mu_Delta = b for a given device right-hand side d_b
 * [n_delta][n_rhs] (CG, MIXED: FP32 sweeps inside FP64 refinement) into
 * d_mu_delta (device).  info as in ddelm_solve (rel_residual: the true FP64
 * |b - S_theta mu| / |b|; ms_total not measured).  Synchronous. */
int ddelm_interface_solve(ddelm_handle *h, const double *d_b, double *d_mu_delta, ddelm_solve_info *info,
                          void *stream);

/* Copies a local block of subdomain `sub` to host memory for inspection
 * (synchronous).  which: 0 K_c^i [m x M], 1 K-bar^i [m x M], 2 A_m^i [nG x M],
 * 3 Lambda^i = A_m^i K^+ E_Gamma [nG x nG], 4 Psi^i = E_Gamma^T K K^+ E_Gamma
 * [nG x nG], 5 Phi^i = A-bar^i K-bar^+ E_Delta [nDl x nDl], 6 S_Pi [n_pi x n_pi]
 * (sub ignored), 7 the four sizes {m, M, nG, nDl} as doubles, 8 the algorithmic
 * flop counts {setup GEMMs, setup Cholesky + inverses, solve GEMMs, tensor-core
 * flops of the MIXED setup, FP64-engine setup flops left in MIXED, the FP32 part
 * of the Cholesky flops, HBM bytes of the BF16 slicing} (sub ignored,
 * out_len >= 5; entries past out_len are not written), 9 the setup plan
 * {scheme, Cholesky passes before the last, setup waves, subdomains per wave,
 * setup graph captured, solve graph captured} (sub ignored, out_len >= 4; the
 * last two when out_len >= 6), 10 V = R^{-1} of the ridge factorisation of
 * [K_c^i; eps I] [M x M], 11 the tile-shape autotuner's outcome {phases timed,
 * phases switched to the other width, their time in ms with the rule's widths,
 * with the chosen widths}, then as far as out_len allows five numbers per phase
 * timed by this handle {phase index, rule's tile width, its ms, alternative
 * width, its ms} (sub ignored, out_len >= 4).  Blocks 0-2 are
 * only kept when the problem was set up with opt.keep_matrices = 1 (which adds
 * their size to the workspace).  out_len is the capacity of host_out in
 * doubles; a block that does not fit returns DDELM_ERR_INVALID_ARG. */
int ddelm_inspect(ddelm_handle *h, int sub, int which, double *host_out, size_t out_len);

/* Per-kernel device timing.  enable = 1 starts recording CUDA events around
 * every launch of the library's kernels (on the launch stream), 0 stops.
 * ms[k] and launches[k] (nullable, DDELM_PROF_CLASSES entries) receive the
 * time and the number of kernel launches accumulated since the last call with
 * reset = 1, per
 * kernel class: 0 feature assembly, 1 FP64 GEMM, 2 Cholesky/inverse,
 * 3 persistent CG, 4 other (gathers, coarse assembly, fills), 5 BF16 slicing
 * of tensor-core GEMM operands, 6 tensor-core (tcgen05) GEMM.  Synchronises
 * on the recorded events. */
#define DDELM_PROF_CLASSES 8
int ddelm_profile(ddelm_handle *h, int enable, int reset, double *ms, long long *launches);

/* Ridge least-squares solve of ONE local ELM system, C = K^+ F (K^+ as in the
 * readings above, eps^2 = eps_rel^2 |K|_F^2 / M), by the library's shifted
 * CholeskyQR3 in FP64, for callers that cannot allocate device memory: code
 * that runs where cudaMalloc is not allowed (inside a host that owns every
 * device allocation, or after the allocator has been locked down) or that is
 * handed only fixed device buffers.  The scratch lives in a file-scope static
 * device array of DDELM_STATIC_SCRATCH_DOUBLES doubles (8 MiB) that every GPU
 * loading the library keeps until the process exits.  Inputs d_K [m x M] and
 * d_F [m x R] (row-major) and the output d_C [M x R] are device buffers owned
 * by the caller.  Limits: 1 <= M <= 256, 1 <= R <= 16, and the call's tables
 * plus its data must fit the array: the data take 2 m M + m R + 8 M^2 + 3 M R
 * + 64 doubles (each of 15 regions rounded up to a multiple of 32), the tables
 * 16 bytes per GEMM output tile (at most 2 ceil(m/64) ceil(M/64) + 5 ceil(M/64)^2
 * + 3 ceil(M/32) tiles) plus about 2.5 KB; sizes beyond that return
 * DDELM_ERR_INVALID_ARG with the reason in ddelm_last_error().  A local matrix
 * whose Cholesky passes meet a pivot that is not positive (K rank deficient
 * with eps_rel = 0) returns DDELM_ERR_RANK_DEFICIENT.  No cudaMalloc, cudaFree
 * or allocating library routine is called.  The first call on a device looks up
 * the array's device address with that device current; make that first call
 * before any stream capture begins.  All calls share the array (it keeps the
 * last call's contents): calls that overlap on the GPU race.  The call blocks
 * until its stream work has completed.  The paper has no counterpart to this
 * entry point. */
#define DDELM_STATIC_SCRATCH_DOUBLES 1048576
int ddelm_local_lstsq_static(const double *d_K, int m, int M, const double *d_F, int R, double eps_rel,
                             double *d_C, void *stream);

void ddelm_destroy(ddelm_handle *h);

const char *ddelm_status_string(int status);

/* The reason behind the last failure on the calling host thread: for
 * DDELM_ERR_CUDA the CUDA error name, message, the failing call and its source
 * location; for a problem that ddelm_query, ddelm_setup or
 * ddelm_local_lstsq_static rejected (DDELM_ERR_INVALID_ARG) "problem rejected: "
 * and the check that failed ("" if none).  The string stays valid until the next failing call. */
const char *ddelm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DDELM_H */
