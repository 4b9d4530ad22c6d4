/*
 * freeform.h -- C ABI of the GB300 (sm_103a) subspace-construction library.
 *
 * The library builds the skinning-eigenmode subspace of FreeForm (reduced-order
 * deformable simulation from particle-based skinning eigenmodes):
 *
 *   rkpm_build        support neighbours and corrected RKPM shape functions
 *                     (Sec. 3.2 "RKPM", Eqs. 6-11)
 *   rkpm_build_twoset the same for the paper's two-set construction: kernel
 *                     centres chosen from quadrature points by farthest-point
 *                     sampling, Gaussian kernels (Supp. Sec. B "RKPM construction")
 *   assemble_hessian  weight-space Neo-Hookean Hessian H_w (Prop. 1) and the
 *                     RKPM mass matrix M (Sec. 3.2, Eq. 14)
 *   eigenmodes        the k lowest generalized eigenpairs of H_w c = lambda M c
 *                     (Sec. 3.2, Eq. 15; Supp. Sec. B "Eigenanalysis")
 *   eigenmodes_batched the three calls for many objects, overlapped on one GPU
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an ff_status; no C++ exception crosses the ABI.  On an
 *   error ff_last_error() returns a message (for FF_ERR_SINGULAR_MOMENT it names
 *   the particle, by its index in the caller's input order).
 * - Array arguments documented "device" are pointers into memory of the
 *   context's device; the library reads them in stream order on the context's
 *   stream (e.g. torch tensor.data_ptr() with the stream from
 *   torch.cuda.current_stream().cuda_stream).  Arguments documented "host" are
 *   ordinary host memory.  The caller owns every buffer it passes; the context
 *   owns every internal device buffer and frees them in ff_destroy.
 * - Calls are state-ordered: rkpm_build (or rkpm_build_twoset), then
 *   assemble_hessian, then eigenmodes; out of order they return FF_ERR_STATE.
 *   A new build discards the previous cloud, matrices and modes.
 * - Calls synchronise the context's stream before returning (results are
 *   ready on return); host outputs are written before return.
 * - Particle order: the library reorders particles internally (by spatial
 *   cell) for locality; every output is returned in the caller's order.
 */
#ifndef FREEFORM_H
#define FREEFORM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ff_ctx ff_ctx;

typedef enum {
  FF_OK = 0,
  FF_ERR_INVALID_ARG = 1,     /* bad size, NULL pointer, non-finite or non-positive input */
  FF_ERR_CUDA = 2,            /* a CUDA runtime call or kernel launch failed */
  FF_ERR_OOM = 3,             /* device allocation failed */
  FF_ERR_SINGULAR_MOMENT = 4, /* a moment matrix M(X_i) has rank < 4 (fewer than four
                                 non-coplanar nodes cover X_i) */
  FF_ERR_NOT_CONVERGED = 5,   /* eigenmodes hit max_iter; outputs hold the last iterate */
  FF_ERR_NUMERIC = 6,         /* NaN/Inf or a breakdown the solver could not recover from */
  FF_ERR_TIMEOUT = 7,         /* the wall-clock budget of ff_eig_opts ran out */
  FF_ERR_STATE = 8            /* calls out of order */
} ff_status;

typedef enum {
  FF_PREC_FP32 = 0,  /* FP32 shape functions (FP64 fallback for ill-conditioned moment
                        matrices), FP32 matrices and iterates, FP64-accumulated Gram
                        products, FP32 dense Rayleigh-Ritz */
  FF_PREC_FP64 = 1   /* FP64 matrices and results: shape functions and assembly sums in
                        double-float (FP32 pairs, ~2^-47 relative), H_w and M stored in
                        FP64; the eigensolver as set by ff_eig_opts.fp32_phase (the
                        preconditioner stays FP32 / BF16) */
} ff_precision;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `precision` is an
 * ff_precision.  On success *out receives the context. */
ff_status ff_create(ff_ctx** out, int device, void* cuda_stream, int precision);

/* Free a context and every device buffer it owns.  NULL is a no-op. */
void ff_destroy(ff_ctx* ctx);

/* Message of the last failed call on this context ("" if none).  The string
 * stays valid until the next call on the context. */
const char* ff_last_error(const ff_ctx* ctx);

/* Library version string, e.g. "freeform-gb300 0.1". */
const char* ff_version(void);

/* ------------------------------------------------------------------ rkpm_build
 * Supp. Sec. B "RKPM construction" + Sec. 3.2 Eqs. 6-11, nodal discretisation:
 * every particle is both an RKPM node p_k and a quadrature point X_i with
 * weight (volume) v_i.  Node k covers X iff ||X - p_k||^2 < a_k^2, the test
 * evaluated in FP64 on the FP32 inputs as ((dx*dx + dy*dy) + dz*dz) < a_k*a_k
 * without fused multiply-add (bit-exact with the oracle).  The raw kernel is the
 * cubic B-spline w(||X - p_k|| / a_k); the correction uses the linear basis.
 *
 *   particles  device, float[n][3] row-major positions (x, y, z)
 *   volumes    device, float[n] quadrature volumes v_i > 0
 *   support    device, float[n] support radii a_k > 0
 *   n          number of particles, 1 <= n <= 2^31 - 1
 *
 * Errors: FF_ERR_INVALID_ARG on NULL pointers, n out of range, or a non-finite
 * position / non-positive volume or radius (message names the first one);
 * FF_ERR_SINGULAR_MOMENT if some moment matrix has rank < 4. */
ff_status rkpm_build(ff_ctx* ctx, const float* particles, const float* volumes,
                     const float* support, int64_t n);

/* ----------------------------------------------------------- rkpm_build_twoset
 * Supp. Sec. B "RKPM construction" with the kernel of Sec. 3.2: two point sets.
 * The n given points are quadrature points X_i with volumes v_i (an inside grid
 * of the object, or its own points).  K kernel centres p_k are chosen among
 * them by farthest-point sampling: the first is point `start`, each next one
 * the point farthest from those chosen, ties to the lowest index.  Centre k has
 * radius r_k = distance to its second-nearest other centre, raw kernel
 * exp(-||X - p_k||^2 / r_k^2) and covers X iff ||X - p_k||^2 < trunc^2 r_k^2
 * (every X when trunc = 0).  Squared distances, their comparisons and r_k are
 * the FP64 values of ((dx*dx + dy*dy) + dz*dz) on the FP32 inputs without fused
 * multiply-add, r_k = sqrt in FP64 (bit-exact with the oracle).  The shape
 * functions (corrected, linear basis, Eqs. 7, 9-10) are evaluated at the
 * quadrature points.  Afterwards the unknowns are the K centres: assemble_hessian
 * takes per-point materials of length n, eigenmodes returns K x k modes in
 * the centres' order of choice, and ff_skinning_weights evaluates the fields
 * with these Gaussian shape functions.  The warm start takes nodal clouds only.
 *
 *   points   device, float[n][3] row-major quadrature points
 *   volumes  device, float[n] quadrature volumes v_i > 0
 *   n        number of points, 4 <= n <= 2^31 - 1
 *   K        number of centres, 4 <= K <= n
 *   trunc    cut radius in units of r_k (> 0), or 0 for the untruncated Gaussian
 *            (every centre at every point: n K pairs)
 *   start    index of the first centre, 0 <= start < n
 *
 * Errors: FF_ERR_INVALID_ARG on NULL pointers, sizes out of range, a
 * non-finite position or non-positive volume (message names the first), or
 * fewer than K distinct positions; FF_ERR_SINGULAR_MOMENT if fewer than four
 * non-coplanar centres cover some quadrature point (message names it). */
ff_status rkpm_build_twoset(ff_ctx* ctx, const float* points, const float* volumes, int64_t n,
                            int32_t K, double trunc, int64_t start);

/* Build precision of the two-set construction in an FF_PREC_FP64 context
 * (applies to the following rkpm_build_twoset calls).  FF_PREC_FP64 (the
 * default): shape functions, material weights and the assembly's sums in
 * double-float (~2^-47).  FF_PREC_FP32: the shape functions in FP32 (the FP64
 * redo for ill-conditioned moment matrices kept) and the sums within a tile of
 * 24 points in FP32, across tiles in FP64 -- assembly in FP32 with FP64-grade
 * dense steps in the eigensolver: H_w and M are
 * still stored in FP64, with about FP32 accuracy (~1e-7 of their entries),
 * and eigenmodes runs as in any FP64 context, its residuals measured against
 * those stored matrices.  FP32 contexts always build in FP32.
 * Errors: FF_ERR_INVALID_ARG for another value, or FF_PREC_FP64 in an FP32
 * context. */
ff_status ff_set_build_precision(ff_ctx* ctx, int precision);

/* The two-set cloud: n_points quadrature points, K centres, centres int64[K]
 * the index of the point chosen as centre k (in the order of choice), radii
 * double[K] the r_k.  Host outputs, any may be NULL; FF_ERR_STATE without a
 * two-set cloud. */
ff_status ff_get_twoset(const ff_ctx* ctx, int64_t* n_points, int32_t* K, int64_t* centres,
                        double* radii);

/* ------------------------------------------------------------ assemble_hessian
 * Prop. 1: (H_w)_kl = sum_i v_i (lambda_i + 4 mu_i) grad phi_k(X_i) . grad phi_l(X_i)
 * Eq. 14:  M_kl     = sum_i v_i phi_k(X_i) phi_l(X_i)
 * with Lame lambda = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu)) at X_i.  The
 * diagonal of H_w is set to minus the sum of its row's off-diagonal entries,
 * so H_w 1 = 0 holds exactly in the stored matrix.
 *
 *   E, nu   device, float[n] per-particle (two-set: per quadrature point)
 *           Young's modulus and Poisson ratio in the caller's order, or NULL to
 *           use the uniform E0 / nu0
 *   E0, nu0 uniform material (used where the array is NULL); E > 0, 0 <= nu < 0.5 */
ff_status assemble_hessian(ff_ctx* ctx, const float* E, const float* nu, double E0,
                           double nu0);

/* ------------------------------------------------------------------ eigenmodes */
typedef struct {
  double tol;           /* stop when every non-constant mode has
                           ||H c - lam M c||_2 / (lam ||M c||_2) <= tol   (1e-6) */
  int max_iter;         /* outer LOBPCG iterations (500) */
  int guard;            /* extra block vectors beyond the k-1 wanted (8) */
  int cheb_degree;      /* degree of the Chebyshev preconditioner; 0 = Jacobi (16) */
  double cheb_ratio;    /* beta / alpha of its interval on D^-1 H (300) */
  uint64_t seed;        /* seed of the random start block (0) */
  double time_budget_s; /* wall-clock budget; <= 0 = none (0) */
  int exclude_constant; /* 1: return k non-constant modes (the paper's m) instead of
                           k modes with the constant mode at index 0 (0) */
  int verbose;          /* print per-iteration residuals to stderr (0) */
  int fp32_phase;       /* FF_PREC_FP64 contexts: 1 = iterate on FP32 roundings of H_w and M
                           until the residual reaches fp32_tol or stops falling, then
                           finish from that block in double-float arithmetic (FP32 pairs,
                           ~2^-47 relative; residuals to tol against the FP64 matrices);
                           0 = FP64 blocks and Rayleigh-Ritz throughout (1) */
  double fp32_tol;      /* residual at which the FP32 phase hands over (1e-4) */
  int cheb_degree_fp64; /* Chebyshev degree of the second phase that follows an FP32 phase;
                           0 = cheb_degree (48) */
  int precond_tc;       /* 1: the preconditioner's H products on tensor cores, with H in
                           BF16 dense tiles of 16-row blocks (block widths 8..120 in steps
                           of 8); 0: sparse FP32 H on CUDA cores (1) */
  int precond_compact;  /* 1: the preconditioner runs on the columns still above tol only,
                           packed to a multiple of 8 (the others are zero either way: the
                           same results, bit for bit on tensor cores, to FP32 rounding of
                           the preconditioned block on CUDA cores); 0: on the whole
                           block (0) */
} ff_eig_opts;

typedef struct {
  int iterations;          /* outer iterations run */
  int converged;           /* modes meeting tol (constant mode counted as converged) */
  int spmm_calls;          /* (H, M) block products in the outer loop */
  int precond_spmv_calls;  /* H block products inside the preconditioner */
  double max_residual;     /* largest relative residual over the non-constant modes */
  double seconds;          /* wall time of the call */
  int warm_start_used;     /* 1 if X0 was used, 0 if the random start was used, 2 if
                              X0 was used, did not converge, and the results come
                              from the random start run after it (the counts and
                              seconds cover both runs) */
  int fp32_iterations;     /* of the iterations, those run in the FP32 phase */
} ff_eig_report;

/* Fill *opts with the defaults listed above. */
void ff_eig_opts_default(ff_eig_opts* opts);

/* The k lowest generalized eigenpairs, ascending.  Constant mode convention
 * (Supp. Sec. B: the spectrum always contains the constant mode with
 * eigenvalue 0): with exclude_constant = 0, index 0 is c0 = 1/sqrt(1^T M 1) * 1
 * with eigenvalue 0, set analytically and deflated; indices 1..k-1 are the
 * lowest non-constant modes.  Modes are M-orthonormal: c^T M c = I.
 *
 *   k        number of modes, 1 <= k <= 256 and k <= n - 1
 *   opts     NULL = defaults
 *   X0       device, optional starting block in the caller's particle order,
 *            column-major n x (m + guard) of the context's precision, m the
 *            number of non-constant modes (k - 1, or k with exclude_constant)
 *            (float for FF_PREC_FP32, double for FF_PREC_FP64); NULL = seeded
 *            random start.  A rank-deficient X0 falls back to the random start,
 *            and so does a start that ends without convergence (not on a
 *            timeout): the solve is then run again from the random start with
 *            the same options, so a start block can cost iterations but never
 *            the answer.
 *   eigvals  host, double[k] eigenvalues (ascending)
 *   modes    device, column-major n x k (leading dimension n) of the context's
 *            precision, in the caller's particle order; may be NULL
 *   rep      host, optional report
 *
 * Returns FF_ERR_NOT_CONVERGED when max_iter is reached or the residual has
 * stopped falling (40 iterations without a new best), FF_ERR_TIMEOUT when the
 * time budget runs out; the outputs then hold the iterate with the smallest
 * largest residual seen. */
ff_status eigenmodes(ff_ctx* ctx, int k, const ff_eig_opts* opts, const void* X0,
                     double* eigvals, void* modes, ff_eig_report* rep);

/* ---------------------------------------------------------- eigenmodes_batched
 * Many objects in one call: for every item, rkpm_build + assemble_hessian +
 * eigenmodes exactly as the single-object calls do them (same kernels, same
 * arithmetic, so each item's results equal those of the three calls on their
 * own).  `workers` host threads (0: min(count, 8)) each drive their own
 * context on their own non-blocking CUDA stream of `device`, taking the
 * objects largest first from a shared counter, so the latency-bound solves of
 * several objects overlap on the GPU.  The call synchronises the device before
 * it starts (the inputs must be ready on any stream) and returns when every
 * item is done.
 *
 *   device, precision  as for ff_create
 *   items     host array of count items; inputs as for rkpm_build and
 *             assemble_hessian, outputs as for eigenmodes (modes may be NULL,
 *             report may be NULL); status and error are written for every item
 *             (error: the item's ff_last_error message, empty when FF_OK)
 *   opts      NULL = defaults; the same options for every item
 *
 * Returns FF_OK when every item succeeded, else the status of the first failed
 * item in array order; FF_ERR_INVALID_ARG on NULL items with count > 0, count
 * < 0, a bad precision or a bad workers count; FF_ERR_CUDA when the device is
 * not usable.  Items no worker could start (every worker failed to create its
 * context) keep FF_ERR_CUDA. */
typedef struct {
  const float* particles;  /* device, float[n][3] */
  const float* volumes;    /* device, float[n] */
  const float* support;    /* device, float[n] */
  int64_t n;
  const float* E;          /* device float[n] or NULL (uniform E0) */
  const float* nu;         /* device float[n] or NULL (uniform nu0) */
  double E0;
  double nu0;
  int k;                   /* modes wanted, as for eigenmodes */
  double* eigvals;         /* host, double[k] */
  void* modes;             /* device, column-major n x k of the precision, or NULL */
  ff_eig_report* report;   /* host, or NULL */
  ff_status status;        /* out */
  char error[192];         /* out */
} ff_batch_item;

ff_status eigenmodes_batched(int device, int precision, ff_batch_item* items, int count,
                             const ff_eig_opts* opts, int workers);

/* ------------------------------------------------------------ host buffers
 * The whole subspace construction from host memory, for callers without
 * device arrays: the inputs are copied to device buffers the context owns (on
 * its stream; pinned host memory makes the copies asynchronous DMA), the
 * three calls run as above, and the eigenvalues and modes are copied back.
 * Arguments as for rkpm_build / rkpm_build_twoset, assemble_hessian and
 * eigenmodes, except that every array is HOST memory:
 *   E, nu    host float[n] per-particle (two-set: per point) material, or NULL
 *            for the uniform E0 / nu0
 *   eigvals  host double[k]
 *   modes    host, column-major n x k (two-set: K x k) of the context's
 *            precision, or NULL
 * Errors: those of the three calls (the first failing call's status); with
 * FF_ERR_NOT_CONVERGED, FF_ERR_TIMEOUT or FF_ERR_NUMERIC the outputs still
 * hold the eigenmodes call's result.  The warm start is not offered here. */
ff_status ff_subspace_host(ff_ctx* ctx, const float* particles, const float* volumes,
                           const float* support, const float* E, const float* nu, int64_t n,
                           double E0, double nu0, int k, const ff_eig_opts* opts,
                           double* eigvals, void* modes, ff_eig_report* rep);
ff_status ff_subspace_twoset_host(ff_ctx* ctx, const float* points, const float* volumes,
                                  const float* E, const float* nu, int64_t n, int32_t K,
                                  double trunc, int64_t start, double E0, double nu0, int k,
                                  const ff_eig_opts* opts, double* eigvals, void* modes,
                                  ff_eig_report* rep);

/* --------------------------------------------------------- inspection exports
 * Copies of the internal results, in the caller's particle order, for parity
 * checks against an independent implementation.  All outputs are host memory. */

/* Sizes after rkpm_build / assemble_hessian: n = unknowns (particles, or the K
 * centres of a two-set cloud), n1 = number of (i, k) support pairs, n2 = stored
 * entries of H_w (= of M), including the diagonal; n2 = 0 before
 * assemble_hessian.  Any pointer may be NULL. */
ff_status ff_get_sizes(const ff_ctx* ctx, int64_t* n, int64_t* n1, int64_t* n2);

/* ------------------------------------------------------------------ skinning weights and LBS */
/* Skinning weight fields at arbitrary points (Sec. 3.2): W^j(X) = sum_k phi_k(X) c_k^j, with
 * phi_k the corrected RKPM shape functions of the built cloud (the kernel, supports and
 * linear basis of rkpm_build, Eqs. 6-11) evaluated at X, and c the nodal values of the
 * fields -- typically the modes eigenmodes returned.
 *   Q    device float[nq * 3] query points, x y z interleaved (any positions the
 *        cloud's supports cover; the particles themselves included)
 *   C    device, context precision, column-major n x m: column j = the nodal values of
 *        field j in the caller's particle order (the layout eigenmodes writes)
 *   W    device, context precision, row-major nq x m output: W[q * m + j] = W^j(Q_q)
 * Needs rkpm_build.  A query point covered by fewer than four non-coplanar nodes (or by
 * none) returns FF_ERR_SINGULAR_MOMENT naming it; m in 1..4096, nq < 2^26. */
ff_status ff_skinning_weights(ff_ctx* ctx, const float* Q, int64_t nq, const void* C, int m,
                              void* W);

/* Linear blend skinning, Eq. 1: x_q = X_q + sum_j W_q^j Z_j [X_q; 1].
 *   Q  device float[nq * 3] rest positions X_q
 *   W  device, context precision, row-major nq x m weights (ff_skinning_weights)
 *   Z  device, context precision, m affine transforms Z_j in R^{3x4}, row-major
 *      (Z[12 j + 4 r + c] = row r, column c of Z_j)
 *   x  device, context precision, nq x 3 output positions
 * Needs a context (any stage); m in 1..4096, nq < 2^26. */
ff_status ff_lbs_deform(ff_ctx* ctx, const float* Q, int64_t nq, const void* W, int m,
                        const void* Z, void* x);

/* Layout of the preconditioner's tensor-core copy of H_w (built by
 * assemble_hessian): row_blocks = ceil(n / 16) blocks of 16 rows, ksteps = the
 * 16-column steps over all blocks' column unions (each step: a 16 x 16 BF16
 * tile of 512 bytes and 16 int32 column indices).  ksteps = 0 when that copy
 * was not built (a block's columns span more than 262144 indices) and the
 * preconditioner runs on the sparse FP32 values.  Any pointer may be NULL. */
ff_status ff_get_precond_layout(const ff_ctx* ctx, int64_t* row_blocks, int64_t* ksteps);

/* Neighbour lists as CSR: ptr int64[rows+1], idx int32[n1] with rows = n (or
 * the n_points quadrature points of a two-set cloud); row i lists the nodes
 * (centres) k covering X_i, ascending.  phi double[n1] and dphi double[3*n1] (x block,
 * then y, then z) are the shape functions phi_k(X_i) and their gradients,
 * aligned with idx; phi / dphi may be NULL. */
ff_status ff_export_rkpm(const ff_ctx* ctx, int64_t* ptr, int32_t* idx, double* phi,
                         double* dphi);

/* Row offsets of the neighbour lists alone: ptr int64[rows+1] as in
 * ff_export_rkpm (rows = n particles in the caller's order, or the n_points
 * quadrature points of a two-set cloud), without copying the lists. */
ff_status ff_export_row_ptr(const ff_ctx* ctx, int64_t* ptr);

/* H_w and M as CSR with ascending columns: row_ptr int64[n+1], col int32[n2],
 * H double[n2], M double[n2].  H or M may be NULL. */
ff_status ff_export_matrices(const ff_ctx* ctx, int64_t* row_ptr, int32_t* col, double* H,
                             double* M);

/* Apply the assembled operators to a block: Y_H = H_w X, Y_M = M X for X
 * column-major n x m in the caller's order (device, context precision).
 * Y_H / Y_M device, same layout; either may be NULL.  1 <= m <= 512. */
ff_status ff_apply_operators(ff_ctx* ctx, const void* X, int m, void* YH, void* YM);

/* Matrix-free application (Prop. 1 and Eq. 14 without assembly): Y_H = H_w X
 * and Y_M = M X computed from the shape-function tables of the built cloud
 * as sum_s G_s^T D G_s X and Phi^T V Phi X, with (G_s)_ik = d_s phi_k(X_i),
 * Phi_ik = phi_k(X_i), D = diag(v_i (lambda_i + 4 mu_i)), V = diag(v_i): one
 * pass per quadrature point (G_s X, Phi X) and one per node over the points it
 * covers (no atomics, fixed summation order).  Needs rkpm_build or
 * rkpm_build_twoset only; the material is given here as for assemble_hessian.
 * It reads the tables instead of the assembled matrices (fewer bytes where a
 * cloud has many more matrix entries than support pairs).  H_w's diagonal is
 * not replaced here: H_w 1 = 0 holds to the rounding of the tables.  FP64
 * sums in FP64 contexts, FP32 otherwise.  A two-set cloud builds its
 * centre -> points lists on the first call (a pass over all points per centre).
 *   E, nu    device float[n] per-particle (two-set: per point) material, or NULL
 *   E0, nu0  uniform material where the arrays are NULL
 *   X        device, column-major n x m in the caller's order, context precision
 *   YH, YM   device, same layout; either may be NULL.  1 <= m <= 512. */
ff_status ff_apply_operators_matfree(ff_ctx* ctx, const float* E, const float* nu, double E0,
                                     double nu0, const void* X, int m, void* YH, void* YM);

/* Allocation-free variant of ff_apply_operators (the paper has no
 * counterpart).  It serves callers that cannot allocate device memory at the
 * time of the call: real-time loops that forbid driver allocations (a
 * cudaMalloc may synchronise the device), processes whose device memory is
 * held by another allocator, or plug-ins given a fixed memory budget.  Same
 * arguments, results and errors as ff_apply_operators, but the three staging
 * panels live in a fixed 32 MiB array in the library's device image (held by
 * every GPU that loads the library until the process exits), and the call
 * makes no cudaMalloc/cudaFree or other allocation.  Requires
 * 3 * n * m * (4 for FF_PREC_FP32, 8 for FF_PREC_FP64) bytes <= 32 MiB (each
 * panel rounded up to 256 bytes); larger blocks return FF_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address.  Like
 * every call of this library it
 * synchronises the context's stream before returning.  All calls share the
 * array: calls that overlap on the GPU race and must be serialised by the
 * caller. */
ff_status ff_apply_operators_noalloc(ff_ctx* ctx, const void* X, int m, void* YH, void* YM);

/* --------------------------------------------------------------- profiling
 * Per-class CUDA-event timing of the library's own launches, recorded on the
 * context stream (off by default; costs two event records per scope). */
typedef enum {
  FF_PROF_PRECOND = 0,        /* Chebyshev preconditioner steps (H-only block products) */
  FF_PROF_SPMM = 1,           /* fused (H_w, M) block products */
  FF_PROF_GRAM = 2,           /* tall-skinny Gram products */
  FF_PROF_RAYLEIGH_RITZ = 3,  /* small dense Rayleigh-Ritz */
  FF_PROF_UPDATE = 4,         /* block updates */
  FF_PROF_BUILD = 5,          /* a whole rkpm_build */
  FF_PROF_ASSEMBLE = 6,       /* a whole assemble_hessian */
  FF_PROF_SETUP = 7,          /* eigensolver set-up: power iteration for the
                                 preconditioner interval */
  FF_PROF_FPS = 8,            /* farthest-point sampling of the two-set centres */
  FF_PROF_COVER = 9,          /* covering lists of the two-set construction */
  FF_PROF_SHAPE = 10,         /* shape-function kernels (the moment solves) */
  FF_PROF_PATTERN = 11,       /* assembly: sparsity pattern of H_w and M */
  FF_PROF_ASM_VALUES = 12     /* assembly: values of H_w and M */
} ff_prof_class;

/* on != 0: reset and start recording; on == 0: stop recording. */
ff_status ff_profile_enable(ff_ctx* ctx, int on);

/* mask != 0: reset and record the classes whose bit (1 << class) is set
 * (a timed run can record one kernel class at two event records per scope
 * without timing the rest); mask == 0: stop recording. */
ff_status ff_profile_classes(ff_ctx* ctx, uint32_t mask);

/* Number of recorded scopes of class `cls` since the last enable and the sum
 * of their durations in milliseconds (synchronises the context stream). */
ff_status ff_profile_read(ff_ctx* ctx, int cls, int64_t* launches, double* total_ms);

/* Number of kernel launches the library has issued in this process. */
int64_t ff_launch_count(void);

/* Self-check of the library's bounded device-side waits (the paper has no
 * counterpart).  The only kernels of the library that wait on other blocks
 * are the farthest-point sampling on the whole GPU (a grid barrier per
 * centre) and the tensor-core Gram (mbarriers); every such wait gives up after
 * a bounded number of clock cycles and reports FF_ERR_TIMEOUT instead of
 * hanging.  This call runs that grid barrier with one arrival missing, so
 * that its wait can only end by running out after wait_cycles SM clock cycles
 * (1e6 .. 4e9; about 2e9 a second at GB300's clock).  Returns FF_ERR_TIMEOUT
 * when the wait ran out and the kernel returned (the expected outcome; the
 * device stays usable), FF_ERR_CUDA when the device has no cooperative launch
 * or a CUDA call failed, FF_ERR_INVALID_ARG on a bad device or wait. */
ff_status ff_selftest_device_wait(int device, int64_t wait_cycles);

/* --------------------------------------------------------- learned warm start
 * The paper starts its LOBPCG from a random block (Supp. Sec. B).  This
 * library can instead start from a block predicted by a small point network
 * from the particle cloud; the eigenproblem (Sec. 3.2, Eq. 15) and its
 * tolerances are unchanged, and a start block that turns out rank-deficient
 * falls back to the random start inside eigenmodes().  The paper has no
 * counterpart of these calls.
 *
 * Features (FF_WS_FEATURES per particle) in the cloud's canonical frame
 * (volume-weighted centroid mu, principal axes R sorted by descending
 * variance with each axis signed so that the third moment along it is >= 0,
 * scale s = sqrt(trace of the covariance)):
 *   0-2   R^T (X_i - mu) / s
 *   3-5   R^T (mean of the support neighbours' positions - X_i) / a_i
 *   6-8   diagonal of R^T C_i R / a_i^2, C_i the neighbours' covariance
 *   9     neighbour count / mean count     10  a_i / s     11  v_i / mean v
 *   12-13 sqrt of the 2nd and 3rd principal variances over the 1st
 *   14    log(n) / 16                      15  1
 * Network (FF_WS_OUTPUTS outputs, 170,784 parameters; BF16 weights and
 * activations, FP32 accumulation; flat FP32 order W1 b1 ... W5 b5, every W
 * row-major [out][in]):
 *   h1 = relu(W1 f + b1) 16->128,  h2 = relu(W2 h1 + b2) 128->256,
 *   g = max over particles of h2,  h3 = relu(W3 [h1; g] + b3) 384->256,
 *   h4 = relu(W4 h3 + b4) 256->128,  y = W5 h4 + b5 128->32.
 * Training loss for a cloud with m known modes C (W = diag(v) / sum v):
 *   L = 1 - trace(K^-1 Z^T G^-1 Z) / m,  G = Y^T W Y + eps I,  Z = Y^T W C,
 *   K = C^T W C,  eps = 1e-6 trace(Y^T W Y) / 32
 * (0 when span(Y) contains span(C), 1 when the spans are W-orthogonal),
 * minimised by Adam (beta1 0.9, beta2 0.999, epsilon 1e-8). */
#define FF_WS_FEATURES 16
#define FF_WS_OUTPUTS 32

typedef struct ff_net ff_net;

/* Number of network parameters (170784). */
int64_t ff_net_num_params(void);

/* Create / destroy a network with its Adam state on a device and stream
 * (NULL stream = the legacy default stream).  Parameters start at zero. */
ff_status ff_net_create(ff_net** out, int device, void* cuda_stream);
void ff_net_destroy(ff_net* net);
/* Message of the last failed call on this network ("" if none). */
const char* ff_net_last_error(const ff_net* net);

/* He-normal weights and zero biases from a seed; resets the Adam state. */
ff_status ff_net_init(ff_net* net, uint64_t seed);
/* Copy the flat FP32 parameters in from / out to host memory; count must be
 * ff_net_num_params().  Setting resets the Adam state. */
ff_status ff_net_set_params(ff_net* net, const float* params, int64_t count);
ff_status ff_net_get_params(ff_net* net, float* params, int64_t count);

/* Features of the context's cloud (after rkpm_build).
 *   feat  device, float[n * FF_WS_FEATURES], row-major per particle, caller order */
ff_status ff_warmstart_features(ff_ctx* ctx, float* feat);

/* Network outputs for one cloud.
 *   feat  device, float[n * FF_WS_FEATURES] (as above);  n >= 1
 *   out   device, float[n * FF_WS_OUTPUTS], row-major per particle */
ff_status ff_net_forward(ff_net* net, const float* feat, int64_t n, float* out);

/* Loss and gradient for one cloud without updating the parameters.
 *   vol    device, float[n] quadrature volumes (caller order)
 *   modes  device, float column-major n x m known modes, 1 <= m <= 32
 *   loss   host, double
 *   grad   host, float[ff_net_num_params()] or NULL */
ff_status ff_net_loss_grad(ff_net* net, const float* feat, const float* vol, int64_t n,
                           const float* modes, int m, double* loss, float* grad);

/* One Adam step on one cloud with learning rate lr; *loss (host, may be NULL)
 * receives the loss before the step. */
ff_status ff_net_train_step(ff_net* net, const float* feat, const float* vol, int64_t n,
                            const float* modes, int m, float lr, double* loss);

/* Start block for eigenmodes(ctx, k, opts, X0, ...): features, the network,
 * and the block's remaining guard columns from opts->seed.
 *   X0  device, column-major n x (m + guard) in the context's precision and the
 *       caller's order (m = k - 1, or k with exclude_constant): the layout
 *       eigenmodes() takes; opts NULL = defaults */
ff_status ff_warmstart_block(ff_ctx* ctx, ff_net* net, int k, const ff_eig_opts* opts,
                             void* X0);

#ifdef __cplusplus
}
#endif

#endif /* FREEFORM_H */
