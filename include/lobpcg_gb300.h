/*
 * lobpcg_gb300.h -- C ABI of the GB300 (sm_103a) LOBPCG eigensolver.
 *
 * Computes the m smallest eigenpairs of the 7-point finite-difference 3-D
 * Laplacian with Dirichlet boundaries by the block Locally Optimal
 * Preconditioned Conjugate Gradient method of Knyazev, Argentati, Lashuk and
 * Ovtchinnikov, "Block Locally Optimal Preconditioned Eigenvalue Xolvers
 * (BLOPEX) in hypre and PETSc": the algorithm of Section 2.2 with B = I, no
 * constraints and the soft locking of Section 2.3, preconditioned by a
 * geometric-multigrid V-cycle that stands in for the paper's hypre/PETSc
 * preconditioners.  Every step of an iteration runs in this library's own
 * CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 *  - Return value: a status code (LOBPCG_OK = 0, LOBPCG_NOT_CONVERGED = 1,
 *    negative = error).  The library never aborts, exits or traps.  A CUDA
 *    error poisons the handle: afterwards every call except lobpcg_destroy
 *    and lobpcg_last_error returns LOBPCG_ERR_CUDA.
 *  - Blocks of vectors are column-major: column j of an n-by-m block starts at
 *    ptr + j*ld (ld >= n, in elements).  Grid point (i, j, k) of an
 *    nx x ny x nz interior grid (0-based) has row index p = i + nx*(j + ny*k).
 *  - "device" pointers are CUDA device (or managed) memory on the handle's
 *    device; "host" pointers are ordinary host memory.  Input pointers are
 *    borrowed for the duration of the call only; output buffers belong to the
 *    caller.  The handle owns all of its workspace.
 *  - All device work is enqueued on the handle's stream.  Entry points that
 *    return host-visible results synchronise that stream before returning.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef LOBPCG_GB300_H
#define LOBPCG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LOBPCG_OK              0
#define LOBPCG_NOT_CONVERGED   1   /* maxit reached; outputs are valid      */
#define LOBPCG_ERR_ARG        -1   /* invalid argument                      */
#define LOBPCG_ERR_OOM        -2   /* the allocator returned NULL           */
#define LOBPCG_ERR_CUDA       -3   /* CUDA error; the handle is poisoned    */
#define LOBPCG_ERR_BREAKDOWN  -4   /* Gram matrix of X or W_J not positive definite */
#define LOBPCG_ERR_NONFINITE  -5   /* NaN or Inf in the iterates            */
#define LOBPCG_ERR_STATE      -6   /* call out of order                     */
#define LOBPCG_ERR_TIMEOUT    -7   /* a bounded wait inside a kernel (an mbarrier of a TMA
                                      ring or of the tensor-core pipeline) gave up; the
                                      kernel recorded it and returned, the handle stays usable */

/* ---- enumerations ------------------------------------------------------ */
#define LOBPCG_FP64            0   /* every step in float64                 */
#define LOBPCG_MIXED           1   /* X, AX, small matrices float64; W / P family float32;
                                      V-cycle float32 with bfloat16 coarse levels; Gram in
                                      float32 with compensated sums; float64 final check */

#define LOBPCG_LAPLACE7        0   /* constant-coefficient 7-point stencil  */
#define LOBPCG_VARCOEF7        1   /* -div(kappa grad u), kappa per face     */

#define LOBPCG_PRECOND_NONE    0   /* T = I                                 */
#define LOBPCG_PRECOND_GMG     1   /* geometric-multigrid V-cycle           */

#define LOBPCG_TOL_RELATIVE    0   /* ||A x_j - l_j x_j|| <= tol * |l_j|    */
#define LOBPCG_TOL_ABSOLUTE    1   /* ||A x_j - l_j x_j|| <= tol            */

#define LOBPCG_GRAM_EXPLICIT   0   /* all Gram blocks computed, symmetrised */
#define LOBPCG_GRAM_PAPER      1   /* Lambda / I diagonal blocks (the Gram blocks as printed) */

#define LOBPCG_MAX_M         100   /* largest block size m (float64 form)   */
#define LOBPCG_MAX_M_MIXED    32   /* largest block size m of the mixed form */
#define LOBPCG_NPHASES         8

/* Phase indices of lobpcg_info.phase_ms. */
#define LOBPCG_PH_RESIDUAL     0   /* residuals and their norms */
#define LOBPCG_PH_PRECOND      1   /* the preconditioning (the V-cycle) */
#define LOBPCG_PH_CHOLQR_W     2   /* the orthonormalisation of W; mixed form: with the Gram-Schmidt of W against X */
#define LOBPCG_PH_SPMV         3   /* the product A W    */
#define LOBPCG_PH_CHOLQR_P     4   /* the orthonormalisation of P; mixed form: with the Gram-Schmidt of P
                                      against [X W] and AP_J = A P_J */
#define LOBPCG_PH_GRAM         5   /* the Gram matrices of the Rayleigh-Ritz basis */
#define LOBPCG_PH_RR           6   /* the Rayleigh-Ritz step    */
#define LOBPCG_PH_UPDATE       7   /* the Ritz update */

typedef struct lobpcg_handle lobpcg_t;

/* Device-memory allocator.  alloc returns device memory usable on `stream`
 * (a cudaStream_t) or NULL; free releases it.  With a NULL allocator the
 * library uses cudaMallocAsync / cudaFreeAsync on the handle's stream. */
typedef struct lobpcg_allocator {
    void* ctx;
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void  (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} lobpcg_allocator;

/* Result summary of a solve. */
typedef struct lobpcg_info {
    int32_t status;          /* same value as the return code                     */
    int32_t iters;           /* iterations performed (k at which J became empty)  */
    int32_t active;          /* |J| at exit                                       */
    int32_t p_dropped;       /* iterations in which the P block was dropped       */
    int32_t fp64_sweeps;     /* float64 confirmations performed: mixed form, correction
                                sweeps; float64 form, final checks (every residual from a
                                fresh A X once J is empty)                         */
    int32_t reserved;
    double  max_rel_resid;   /* max_j ||A x_j - l_j x_j|| / |l_j|, from A X at exit */
    double  setup_ms;        /* device time of the set-up                           */
    double  solve_ms;        /* device time of the iteration loop                  */
    int64_t kernel_launches; /* kernels this library launched during the call       */
    double  phase_ms[LOBPCG_NPHASES];  /* device time per phase, summed over iterations;
                                          filled only when phase timing is enabled */
} lobpcg_info;

/* ---- solver-level entry points ------------------------------------------ */

/* Create a handle on CUDA device `device`.  `stream` is a cudaStream_t (NULL =
 * the legacy default stream); `alloc` may be NULL; `precision` is LOBPCG_FP64
 * or LOBPCG_MIXED.  In the mixed form, once every implicit residual passes the
 * tolerance, a float64 correction sweep (the initial orthonormalisation and Rayleigh-Ritz step of the algorithm on the
 * current X with a float64 A X) recomputes the Ritz pairs and their residuals;
 * columns that still fail re-enter the iteration (at most 16 sweeps; then the
 * solve returns LOBPCG_NOT_CONVERGED).
 * On success *h receives the handle.  Errors: ERR_ARG, ERR_CUDA. */
int lobpcg_create(lobpcg_t** h, int device, void* stream,
                  const lobpcg_allocator* alloc, int precision);

/* Set the operator A.  kind = LOBPCG_LAPLACE7 (Section 4, model problem):
 * (A u)_p = scale * (6 u_p - sum of the six neighbours of p), neighbours
 * outside the grid are zero; scale > 0 (h^-2 = (n+1)^2 for the unit cube; 1.0
 * gives the unscaled spectrum of Section 4.1); kappa_faces must be NULL.
 * kind = LOBPCG_VARCOEF7 (the differentiated operator -div(kappa grad u), unit
 * spacing, Dirichlet): (A u)_p = scale * sum over the six faces f of p of
 * kappa_f (u_p - u_q), u_q = 0 outside; kappa_faces points to the face
 * coefficients (host or device, float64, copied): (nx+1)*ny*nz x-faces, face
 * (f, j, k) between cells (f-1, j, k) and (f, j, k), then nx*(ny+1)*nz y-faces,
 * then nx*ny*(nz+1) z-faces, x fastest in each part; all > 0.  VARCOEF7 needs a
 * LOBPCG_FP64 handle.  nx, ny, nz >= 1.  Resets the preconditioner.
 * Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
int lobpcg_set_operator(lobpcg_t* h, int kind, int nx, int ny, int nz,
                        double scale, const double* kappa_faces);

/* Set the preconditioner T (Section 2.2; Section 2.1.1 requires T linear,
 * symmetric, positive definite).  kind = LOBPCG_PRECOND_NONE or _GMG.  For GMG:
 * `levels` >= 1 grid levels, level l+1 having floor(n/2) points per axis;
 * nu_pre = nu_post >= 1 weighted-Jacobi sweeps with weight omega in (0, 1];
 * full-weighting restriction R = P^T/8, trilinear prolongation P, rediscretised
 * coarse operators (scale / 4 per level) and an exact dense solve on the
 * coarsest level (at most 4096 points).  Must follow lobpcg_set_operator.
 * Errors: ERR_ARG, ERR_STATE, ERR_OOM, ERR_CUDA. */
int lobpcg_set_preconditioner(lobpcg_t* h, int kind, int levels, int nu_pre,
                              int nu_post, double omega);

/* Options: tolerance mode (LOBPCG_TOL_*), Gram variant (LOBPCG_GRAM_*), and
 * per-phase device timing (0/1; adds event records inside each iteration). */
int lobpcg_set_options(lobpcg_t* h, int tol_mode, int gram_mode, int phase_timing);

/* Inner PCG preconditioning (the paper's Section 4.2, "Performance Versus the
 * Number of Inner Iterations"): the preconditioning applies T = k iterations of
 * preconditioned conjugate gradients for A E = W_J from E = 0, preconditioned by
 * the preconditioner set with lobpcg_set_preconditioner, each column an
 * independent solve (float64; a column stops early only if p^T A p <= 0 or
 * r^T z <= 0).  iters = 0 (default) applies the preconditioner directly.  T is
 * then a nonlinear map, which LOBPCG tolerates.  lobpcg_op_precond applies the
 * same T.  Returns ERR_ARG for iters < 0 or > 10000, or iters > 0 on a
 * LOBPCG_MIXED handle. */
int lobpcg_set_inner_pcg(lobpcg_t* h, int iters);

/* Engine of the Gram products.
 * Float64 form (and the float64 steps of the mixed form): unless the engine is
 * LOBPCG_ENGINE_SIMT, the Gram matrices of the Rayleigh-Ritz basis (and those of
 * lobpcg_op_gram) with at most 48 columns run on the tensor cores by error-free
 * digit products (the Cholesky Grams of single blocks, whose factor decides a
 * breakdown, stay on the float64 pipe): per window of 1024 grid points every
 * column is split into 8 signed 7-bit digits under the window's largest
 * exponent (bfloat16, exact), the digit-pair products are summed exactly by
 * tcgen05 MMAs in float32 tensor memory, and the pairs are combined in 64-bit
 * integers and added in float64 (Ozaki, Ogita and Oishi's error-free splitting;
 * about 2^-48 of the window's largest products, float64 quality for smooth
 * grid functions).  LOBPCG_ENGINE_SIMT keeps the float64 FMA pipe.
 * Mixed form, float32 Gram products (the orthonormalisations of W and P and the Gram matrices; the double-float
 * X^T X block is unaffected):
 *   LOBPCG_ENGINE_TENSOR: tcgen05 tensor-core MMAs on 3 x TF32 splits (hi*hi +
 *     hi*lo + lo*hi, about 2^-21 relative per product), float32 accumulation
 *     in tensor memory over at most 128 grid points (the tensor cores round it
 *     toward zero: about 1e-6 relative to |s_i| |s_j| when the stacked blocks
 *     have at most 128 columns, 3e-6 up to 192), compensated float32 sums of
 *     those, float64 chunk sums.  Used whenever the stacked blocks fit (each
 *     block padded to a multiple of 8 columns, at most 192 in all, the left
 *     operands within the first 128); otherwise the SIMT engine runs.
 *   LOBPCG_ENGINE_SIMT: float32 products with compensated float32 sums on the
 *     CUDA cores (about 2^-24 relative per product).
 *   LOBPCG_ENGINE_AUTO (default): the tensor cores for stacks of more than 64
 *     columns (the residual-form Gram), the SIMT engine below that.  A tensor
 *     core MMA costs about the same for any N <= 256 on GB300, so the tensor
 *     form pays off only for wide stacks.
 * Returns ERR_ARG for an unknown engine. */
#define LOBPCG_ENGINE_AUTO     0
#define LOBPCG_ENGINE_SIMT     1
#define LOBPCG_ENGINE_TENSOR   2
int lobpcg_set_gram_engine(lobpcg_t* h, int engine);

/* Failure detection: the float32 kernels of the mixed form that stream their
 * inputs through a ring of shared-memory stages filled by the Tensor Memory
 * Accelerator (the SIMT Gram tiles and the streamed block products) wait for
 * each stage on an mbarrier, and every such wait is bounded: after `polls`
 * unsuccessful polls it gives up, the kernel waits (with its own, unchanged
 * bound) for the copies it still has in flight, records the failure and
 * returns, and the call returns LOBPCG_ERR_TIMEOUT with the handle still
 * usable.  polls < 0 restores the default bound (2^22 polls, seconds); polls =
 * 0 makes every such wait give up at once, which lets a caller exercise its
 * handling of LOBPCG_ERR_TIMEOUT without a hung GPU.  The tensor-core Gram
 * engine keeps its fixed bounds.  Never returns an error for a valid handle. */
int lobpcg_set_wait_limit(lobpcg_t* h, int polls);

/* Constraints, the hard locking of the paper's Section 2.3 (the constraint projections of
 * Section 2.2's algorithm): Y is an n-by-l block (column j at Y + j * ldy, float64, device memory,
 * or host memory if on_host != 0) of l linearly independent columns; it is
 * copied.  The following solves work in the complement of span(Y): the constraint projection of X
 * projects the initial block, X = X - Y (Y^T Y)^-1 (Y^T X), and the constraint projection of W every
 * preconditioned residual block, W_J = W_J - Y (Y^T Y)^-1 (Y^T W_J) (B = I), so
 * with the eigenvectors of earlier solves as Y a solve continues the spectrum
 * (the repeated calls the paper recommends for many eigenpairs).  The library
 * applies the same projector through an orthonormal basis of span(Y), built
 * at the next solve in float64 (block Gram-Schmidt and Cholesky QR, twice); the
 * mixed form projects its float32 W_J twice against a float32 copy and
 * re-projects X in float64 before each float64 sweep.  l = 0 removes the
 * constraints.  Returns ERR_ARG for l < 0, 2 l >= n, a NULL Y with l > 0 or
 * ldy < n; the next solve returns ERR_ARG if 2 (m + l) > n and ERR_BREAKDOWN
 * if Y^T Y is not numerically positive definite. */
int lobpcg_set_constraints(lobpcg_t* h, const double* Y, int l, int64_t ldy,
                           int on_host);

/* Supply the initial block X0 (Algorithm input X): n-by-m, column-major, leading
 * dimension ldx, copied into the handle.  on_host = 1: X0 is host memory;
 * 0: device memory.  Used by the next lobpcg_solve / lobpcg_begin with the same
 * m instead of the seeded random block.  Errors: ERR_ARG, ERR_STATE, ERR_CUDA. */
int lobpcg_set_initial(lobpcg_t* h, const double* X0, int m, int64_t ldx, int on_host);

/* Solve: the set-up, then iterations k = 0..maxit of the iteration of Section 2.2 until every
 * column satisfies the tolerance (the pass k = maxit performs only the residuals and the soft-locking test).
 * Soft-locked columns stay in the Rayleigh-Ritz basis (Section 2.3), so a
 * locked column can drift above the tolerance; when J is empty the float64
 * form therefore recomputes every residual from a fresh A X (which replaces
 * the implicitly updated AX) and returns the failing columns to J, and the
 * mixed form runs its float64 correction sweep.  The solve converges only when
 * that check passes: on LOBPCG_OK every residual meets the tolerance.
 * Without lobpcg_set_initial, X0 is the seeded SplitMix64 block: entry
 * (p, j) = 2 * (out[p + n j] >> 11) * 2^-53 - 1, out = outputs of SplitMix64
 * started at state `seed`.  1 <= m <= LOBPCG_MAX_M, m <= n/2; tol >= 0;
 * maxit >= 0.  `out` may be NULL.  Returns OK, NOT_CONVERGED, ERR_BREAKDOWN,
 * ERR_NONFINITE, ERR_ARG, ERR_STATE, ERR_OOM or ERR_CUDA.  After OK or
 * NOT_CONVERGED (and after BREAKDOWN / NONFINITE, with the last valid
 * iterate) lobpcg_get_eigenpairs returns the result. */
int lobpcg_solve(lobpcg_t* h, int m, double tol, int maxit, uint64_t seed,
                 lobpcg_info* out);

/* Step-wise form of lobpcg_solve.  lobpcg_begin performs the set-up;
 * lobpcg_iterate then performs up to `steps` passes of the iteration of Section 2.2 and returns
 * OK once J is empty (NOT_CONVERGED while columns remain active).  A tol of 0
 * keeps every column active (fixed work per pass).  lobpcg_finish recomputes
 * the residuals from A X (as lobpcg_solve does at exit). */
int lobpcg_begin(lobpcg_t* h, int m, double tol, uint64_t seed);
int lobpcg_iterate(lobpcg_t* h, int steps, lobpcg_info* out);
int lobpcg_finish(lobpcg_t* h, lobpcg_info* out);

/* Copy out the result: lambda (host, m values ascending), X (n-by-m,
 * column-major, leading dimension ldx; host if x_on_host else device; may be
 * NULL) and resid (host, m values of ||A x_j - lambda_j x_j||_2 from A X; may
 * be NULL).  Errors: ERR_STATE (nothing solved yet), ERR_ARG, ERR_CUDA. */
int lobpcg_get_eigenpairs(lobpcg_t* h, double* lambda, double* X, int64_t ldx,
                          int x_on_host, double* resid);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle.  h may be NULL: then the last error of a handle-free call
 * (lobpcg_create, lobpcg_gram_noalloc) on the calling thread. */
const char* lobpcg_last_error(const lobpcg_t* h);

/* Release the handle and all of its workspace.  NULL is accepted. */
int lobpcg_destroy(lobpcg_t* h);

/* Eigenvalue gradient of the variable-coefficient operator (LOBPCG_VARCOEF7)
 * for the finished solve: grad_faces[f] = sum_j w[j] d lambda_j / d kappa_f =
 * scale * sum_j w[j] (x_j,q - x_j,p)^2 over the m computed unit eigenvectors
 * (x_j,q = 0 outside the box), the first-order perturbation of a simple
 * eigenvalue; with equal weights over a cluster of equal eigenvalues the sum is
 * independent of the basis chosen inside the cluster.  w: host array of m
 * weights; grad_faces: device array in the kappa_faces layout.  Errors: ERR_ARG,
 * ERR_STATE (no finished solve, or another operator kind), ERR_CUDA. */
int lobpcg_eig_grad_kappa(lobpcg_t* h, const double* w, double* grad_faces);

/* ---- kernel-level entry points -------------------------------------------
 * Each applies one step of the iteration to caller-owned device buffers, on
 * the handle's stream, using the handle's operator and preconditioner.  They
 * exist so that every kernel can be checked on its own and reused. */

/* X0 generator (Algorithm input; SplitMix64 as in lobpcg_solve): writes the
 * n-by-m block with n = the operator's point count into device X. */
int lobpcg_op_random_block(lobpcg_t* h, uint64_t seed, int m, double* X, int64_t ldx);

/* Y = A X for `ncols` columns (Section 2.2): device X, Y, which
 * must not overlap. */
int lobpcg_op_stencil(lobpcg_t* h, int ncols, const double* X, int64_t ldx,
                      double* Y, int64_t ldy);

/* The mixed form's SpMV (Section 2.2, on a LOBPCG_MIXED handle): Y = A X
 * for ncols float32 device columns (n rows, leading dimensions ldx, ldy >= n),
 * float32 arithmetic, each point's six neighbour differences summed before the
 * scaling.  X and Y must not overlap.  ERR_ARG on a LOBPCG_FP64 handle. */
int lobpcg_op_stencil_f32(lobpcg_t* h, int ncols, const float* X, int64_t ldx,
                          float* Y, int64_t ldy);

/* E = T R for `ncols` columns (Section 2.2; T = I copies): device R, E,
 * which must not overlap.  Needs a LOBPCG_FP64 handle. */
int lobpcg_op_precond(lobpcg_t* h, int ncols, const double* R, int64_t ldr,
                      double* E, int64_t lde);

/* The mixed form's preconditioner (Section 2.2, on a LOBPCG_MIXED handle):
 * E = T R for ncols float32 device columns (n rows, leading dimensions ldr, lde
 * >= n), the V-cycle with float32 arithmetic on every level, float32 storage on
 * the finest and bfloat16 storage on the coarser levels.  ERR_ARG on a
 * LOBPCG_FP64 handle. */
int lobpcg_op_precond_f32(lobpcg_t* h, int ncols, const float* R, int64_t ldr,
                          float* E, int64_t lde);

/* Column residuals (Section 2.2): for t < ncols, j = cols[t] (host array),
 * W[:, t] = AX[:, j] - lambda[j] X[:, j] (lambda: device, m values) and
 * norms[t] = ||W[:, t]||_2 (host output).  W may be NULL (norms only). */
int lobpcg_op_residual(lobpcg_t* h, int ncols, const int* cols, const double* X,
                       const double* AX, int64_t ld, const double* lambda,
                       double* W, int64_t ldw, double* norms);

/* Gram matrices (Section 2.2): S = [S0 S1 S2] with widths w0, w1, w2
 * (w1, w2 may be 0), each block n rows with leading dimension ld; AS likewise.
 * Writes the q-by-q (q = w0 + w1 + w2) column-major device matrices gramB = S^T S
 * and gramA with the block structure printed in Section 2.2: block (I, J) =
 * S_I^T AS_J for I < J, its transpose below the diagonal, and (S_I^T AS_I +
 * AS_I^T S_I)/2 on the diagonal.  AS0 may be NULL (gramA skipped).  The
 * handle's Gram engine applies (tensor-core digit products for q <= 48 unless
 * LOBPCG_ENGINE_SIMT).  Deterministic: partial sums per thread block are added
 * in a fixed order.  Errors: ERR_ARG, ERR_TIMEOUT, ERR_CUDA. */
int lobpcg_op_gram(lobpcg_t* h, const double* S0, const double* S1, const double* S2,
                   const double* AS0, const double* AS1, const double* AS2,
                   int64_t ld, int w0, int w1, int w2, double* gramA, double* gramB);

/* Float64 Ritz update (Section 2.2): with S = [S0 S1 S2] (widths w0,
 * w1, w2; w1, w2 may be 0; n rows, leading dimension ld >= n) and the
 * q-by-m coefficients C (q = w0 + w1 + w2, column-major, leading dimension q,
 * device), writes Xout = S C and, if Pout != NULL, Pout = S1 C1 + S2 C2 (the
 * rows of C below w0), m columns each with leading dimension ld.  Xout may be
 * S0 and Pout may be S2 (in place).  Unless the engine is LOBPCG_ENGINE_SIMT,
 * products with q <= 32 and at most 28 outputs (2m with Pout, m without) run on
 * the tensor cores by error-free digit products: every grid point split into 8
 * signed 7-bit bfloat16 digits under its largest exponent over the q columns,
 * every column of C under its own, the digit levels s + t <= 8 summed exactly in
 * float32 tensor memory and combined in 64-bit integers (error per output below
 * (q + 4) 2^-54 max_k |S(p, k)| max_k |C(k, j)| plus the final rounding; needs
 * an even ld and 16-byte aligned blocks); otherwise float64 FMAs.  The solver's
 * own calls (the V R^-1 products of lobpcg_op_cholqr and of the iteration, and
 * the update) first scale the columns of S by powers of two (from the rows of
 * R^-1, or from the column maxima of the preceding Gram), so that badly scaled
 * columns keep their relative accuracy.  Errors: ERR_ARG, ERR_TIMEOUT,
 * ERR_CUDA. */
int lobpcg_op_update(lobpcg_t* h, const double* S0, const double* S1, const double* S2,
                     int64_t ld, int w0, int w1, int w2, int m, const double* C,
                     double* Xout, double* Pout);

/* Cholesky orthonormalisation (Section 2.2): G = V^T V,
 * R = chol(G) computed on the unit-diagonal scaling of G, V <- V R^-1 and, if
 * AV != NULL, AV <- AV R^-1 (in place, device, b columns, leading dimension ld).
 * Returns ERR_BREAKDOWN (buffers untouched) if a pivot of the scaled factor is
 * <= b * 2^-52. */
int lobpcg_op_cholqr(lobpcg_t* h, int b, double* V, double* AV, int64_t ld);

/* Mixed form, float32 Gram products (Section 2.2, and the block
 * Gram-Schmidt projections of W and P that the mixed form adds): with float32
 * device blocks S0 (w0 columns), S1 (w1 columns, may be NULL when w1 = 0) and V
 * (b columns), each n rows with the common leading dimension ld (a multiple of
 * 4; pointers 16-byte aligned), writes C = [S0 S1]^T V ((w0 + w1)-by-b,
 * column-major, ld w0 + w1; skipped if C is NULL or w0 + w1 = 0) and
 * G = V^T V (b-by-b, symmetric; skipped if NULL), both float64 on the device.
 * Float32 products, compensated float32 sums, float64 partial sums added in a
 * fixed order.  w0 + w1 <= 2 * LOBPCG_MAX_M, b <= LOBPCG_MAX_M. */
int lobpcg_op_gram_f32(lobpcg_t* h, const float* S0, int w0, const float* S1, int w1,
                       const float* V, int b, int64_t ld, double* C, double* G);

/* Mixed form, Gram matrices in residual form (Section 2.2): basis
 * S = [X W P] with X given as float32 planes (X = Xh + Xl), W (b columns) and
 * P (bp columns, bp = 0: no P block), and T = [R AW AP] with R = AX - X Lambda
 * (Lambda = diag(lambda), lambda: device, m values); all float32 device blocks,
 * n rows, common leading dimension ld (a multiple of 4, 16-byte aligned).
 * Writes gramB = S^T S and gramA = S^T (AS) (q-by-q, q = m + b + bp,
 * column-major, device) with X^T AX = (X^T X) Lambda + X^T R symmetrised,
 * (AX)^T S_j = Lambda X^T S_j + R^T S_j, the upper block triangle S_I^T AS_J of
 * the W / P part (I < J) and (S_I^T AS_I + AS_I^T S_I) / 2 on its diagonal
 * blocks.  X^T X in double-float arithmetic (hi * hi products exact, about
 * 2^-44 relative), all other products float32 with compensated sums. */
int lobpcg_op_gram_residual(lobpcg_t* h, const float* Xh, const float* Xl, const float* W,
                            const float* P, const float* R, const float* AW, const float* AP,
                            int64_t ld, int m, int b, int bp, const double* lambda,
                            double* gramA, double* gramB);

/* Rayleigh-Ritz (Section 2.2) on device matrices: gramA C = gramB C Lambda
 * for q-by-q symmetric gramA, gramB (column-major), the m smallest eigenvalues
 * ascending into device lambda and the gramB-orthonormal eigenvectors into
 * device C (q-by-m, column-major, ld q).  q <= 3 * LOBPCG_MAX_M.  Returns
 * ERR_BREAKDOWN if gramB is not numerically positive definite. */
int lobpcg_op_rayleigh_ritz(lobpcg_t* h, int q, int m, const double* gramA,
                            const double* gramB, double* lambda, double* C);

/* ---- allocation-free entry point -----------------------------------------
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory -- code running inside a host callback or signal
 * handler, an application whose memory pool owns every byte of the device and
 * forbids libraries to allocate, a latency-critical loop where an allocation
 * could stall, or any caller without a handle (a handle allocates workspace).
 *
 * lobpcg_gram_noalloc computes what lobpcg_op_gram computes (gramA and gramB of
 * S = [S0 S1 S2], widths w0, w1, w2, n rows, common leading dimension ld; AS0 =
 * NULL skips gramA) without a handle
 * and without allocating: its per-block partial sums go to one fixed array of
 * 8 MiB of device memory that each GPU loading this library holds until the
 * process exits.  All pointers are device pointers; the work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call returns
 * without waiting for it.  Limit: q = w0 + w1 + w2 <= 96, else LOBPCG_ERR_ARG.
 * No cudaMalloc, cudaFree or other allocating routine is called.  The first
 * call on a device looks up the array's device address and caches it; make that
 * first call before any stream capture.  The cached address belongs to the
 * device's primary context and stays valid for that context's lifetime: a
 * process that resets the device (cudaDeviceReset) must not call this entry
 * point on that device afterwards.  Every call reuses the same array: calls
 * whose kernels may overlap on the GPU (unordered streams or threads) race and
 * give wrong results, so order them.  Errors: LOBPCG_ERR_ARG, LOBPCG_ERR_CUDA;
 * the message is returned by lobpcg_last_error(NULL) on the calling thread. */
int lobpcg_gram_noalloc(const double* S0, const double* S1, const double* S2,
                        const double* AS0, const double* AS1, const double* AS2,
                        int64_t n, int64_t ld, int w0, int w1, int w2,
                        double* gramA, double* gramB, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LOBPCG_GB300_H */
