// Shared definitions of the GB300 LOBPCG library: error type, grid geometry, storage types,
// column lists and the host-side launchers of every kernel.  Kernels live in k_stencil.cu
// (stencil family + V-cycle), k_block.cu (tall-skinny block ops) and k_dense.cu (small dense
// factorizations on one thread block).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <stdexcept>
#include <string>

#include "../../include/lobpcg_gb300.h"

namespace lg {

extern std::atomic<long long> g_kernel_launches;
// Poll limit of the stage waits of the TMA-staged float32 kernels for the calling thread's
// current call (set from the handle for the duration of each call; < 0: the default).
extern thread_local int g_wait_limit;

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& msg) : std::runtime_error(msg), code(c) {}
};

#define LG_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            throw ::lg::Error(LOBPCG_ERR_CUDA, std::string(#call) + ": " +             \
                                                   cudaGetErrorString(e_));            \
    } while (0)
// Every kernel launch of the library is followed by LG_CHECK_LAUNCH, which also counts it.
#define LG_CHECK_LAUNCH()                                                              \
    do {                                                                               \
        ::lg::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);               \
        LG_CUDA(cudaGetLastError());                                                   \
    } while (0)
#define LG_REQUIRE(cond, code, msg)                                                    \
    do {                                                                               \
        if (!(cond)) throw ::lg::Error((code), (msg));                                 \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kMaxM = LOBPCG_MAX_M;
constexpr int kMaxQ = 3 * LOBPCG_MAX_M;   // Rayleigh-Ritz basis [X W_J P_J]
constexpr int kMaxMMixed = LOBPCG_MAX_M_MIXED;
constexpr int kNumSMs = 152;              // GB300: 2 dies x 76 SMs

// Interior grid of one multigrid level; point p = i + nx*(j + ny*k).
struct Grid3 {
    int nx, ny, nz;
    __host__ __device__ int64_t n() const { return (int64_t)nx * ny * nz; }
};

// Up to kMaxM column indices, passed by value as a kernel parameter.
struct ColList {
    int n;
    int idx[kMaxM];
};

// Device status word bits, written by kernels and read with the residual norms.
enum StatusBits : unsigned {
    ST_W_BREAKDOWN = 1u,      // chol(W_J^T W_J) failed (the orthonormalisation of W)
    ST_P_DROPPED = 2u,        // P block dropped this iteration (chol of P or gramB failed)
    ST_RR_BREAKDOWN = 4u,     // gramB not positive definite without P
    ST_X_BREAKDOWN = 8u,      // chol(X^T X) failed (the orthonormalisation of X)
    ST_NONFINITE = 16u,       // non-finite value in a small dense matrix
    ST_TIMEOUT = 32u,         // a bounded wait of a kernel gave up (its results are invalid)
    ST_TIMEOUT_MMA = 64u,     // the tensor-core Gram's wait for its issued MMAs gave up as well
};

// Storage types of the blocks: float64 (FP64 form; X and AX of the mixed form), float32 (the
// W / P family and level 0 of the V-cycle in the mixed form), bfloat16 (coarse V-cycle levels
// of the mixed form).  Arithmetic is float64 on float64 data and float32 otherwise.
enum DType : int { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2 };
inline size_t dtype_size(DType t) { return t == DT_F64 ? 8 : (t == DT_F32 ? 4 : 2); }

// ---------------------------------------------------------------- stencil family
// y = a*x + b*(sum of the 6 neighbours of x) [+ c*z], per column, zero outside the grid;
// x, z and y share the storage type t.
void launch_stencil_axpby(const Grid3& g, int ncols, DType t, double a, double b, const void* x,
                          int64_t ldx, double c, const void* z, int64_t ldz, void* y,
                          int64_t ldy, cudaStream_t st);
// Full-weighting restriction rc = P^T rf / 8 (fine grid gf, type tf -> coarse grid gc, type tc).
void launch_restrict(const Grid3& gf, const Grid3& gc, int ncols, DType tf, const void* rf,
                     int64_t ldf, DType tc, void* rc, int64_t ldc, cudaStream_t st);
// Trilinear prolongation with correction: ef += P ec.
void launch_prolong_add(const Grid3& gf, const Grid3& gc, int ncols, DType tc, const void* ec,
                        int64_t ldc, DType tf, void* ef, int64_t ldf, cudaStream_t st);
// Exact coarsest-level solve e = A_c^-1 r through the discrete sine transform (float64
// arithmetic for every storage type).  `tables` holds the three normalised 1-D sine matrices
// and the eigenvalues (layout from coarse_tables_size / launch_coarse_setup).
int64_t coarse_tables_size(const Grid3& g);
void launch_coarse_setup(const Grid3& g, double scale, double* tables, cudaStream_t st);
void launch_coarse_solve(const Grid3& g, int ncols, DType t, const double* tables, const void* r,
                         int64_t ldr, void* e, int64_t lde, cudaStream_t st);
// The V-cycle on the levels g[0..nl-1] (g[0] the finest of them, scales[l] their operator scales,
// tables = the sine-transform tables of g[nl-1]) in one kernel, one block per column, all level
// vectors in shared memory: e = T r for ncols columns of type t (input and output only touch
// global memory).  For levels of at most kFuseMaxPoints points.
constexpr int kFuseMaxPoints = 4096;
constexpr int kFuseMaxLevels = 12;
size_t vcycle_small_smem(const Grid3* g, int nl, DType t);
void launch_vcycle_small(const Grid3* g, const double* scales, int nl, double omega, int nu_pre, int nu_post,
                         const double* tables, int ncols, DType t, const void* r, int64_t ldr, void* e,
                         int64_t lde, cudaStream_t st);
// Copy (with conversion) of ncols columns of n entries.
void launch_convert(int64_t n, int ncols, DType ts, const void* src, int64_t lds, DType td,
                    void* dst, int64_t ldd, cudaStream_t st);

// ---------------------------------------------------------------- block ops
void launch_random_block(uint64_t seed, int64_t n, int m, double* X, int64_t ldx,
                         cudaStream_t st);
// Partial sums of squares of W[:, t] = AX[:, cols[t]] - lambda[cols[t]] * X[:, cols[t]]
// (float64 arithmetic); writes W (type tw) if non-null.  partial has nchunks * cols.n doubles.
int residual_chunks(int64_t n);
void launch_residual(int64_t n, const ColList& cols, const double* X, const double* AX,
                     int64_t ld, const double* lambda, DType tw, void* W, int64_t ldw,
                     double* partial, cudaStream_t st);
// norms[t] = sqrt(sum_c partial[t*nchunks + c]) in a fixed order.
void launch_norms_finalize(int ncols, int nchunks, const double* partial, double* norms,
                           cudaStream_t st);

// Block pointers of a basis [B0 B1 B2] (widths w[k], common leading dimension in elements).
// Block 0 has storage type t0 (X or AX), blocks 1 and 2 type t12 (the W and P families).
struct Blocks3 {
    const void* p[3];
    int w[3];
    int64_t ld;
    DType t0, t12;
    __host__ __device__ int q() const { return w[0] + w[1] + w[2]; }
};
// Gram partial sums over `nparts` row ranges: part has nparts * 2*q*q doubles; float64 blocks
// and arithmetic (the float32 Grams of the mixed form are in k_gram32.cu).
int gram_parts(int64_t n, int q);
int64_t gram_scratch_doubles(int64_t n, int q);
void launch_gram(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int nparts,
                 cudaStream_t st);
// The same partial sums (float64 blocks of at most 48 columns) on the tensor cores by error-free
// bfloat16 digit products (k_gram_oz.cu); returns the number of row ranges (partials) written,
// 0 if the scratch cannot hold them (nothing launched).
bool gram_oz_fits(int q);
// colmax (device, may be null): the largest exponent field of every column of S, then of AS, over
// all grid points.
int launch_gram_oz(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int64_t part_doubles,
                   unsigned* status, cudaStream_t st, int* colmax = nullptr);
// Y = S C on the tensor cores by error-free bfloat16 digit products (k_tsmm_oz.cu), float64
// blocks of at most 32 columns: output j < nx is S C(:, j) (to out0 + j ldout), output nx + j
// (j < np) is the sum over rows k >= w0p of S(:, k) C(k, j) (to out1 + j ldout); C is q x nx,
// column-major, leading dimension ldc, on the device.  Outputs may overwrite S in place.
// Column k of S is scaled by 2^a_k and row k of C by 2^-a_k before the split (exact; the digit
// frame of a grid point is then its largest scaled entry): TZ_SCALE_NONE a_k = 0;
// TZ_SCALE_C_ROWS 2^a_k about the largest |C(k, .)| (V R^-1: equilibrates the columns of V);
// TZ_SCALE_S_COLS 2^-a_k about the largest |S(., k)|, from sexp (device, the largest exponent
// field of each column of S, e.g. from launch_gram_oz).
// Skipped if *status & skip; a bounded wait that gives up sets ST_TIMEOUT.  Returns false
// (nothing launched) for shapes outside the kernel's limits.
enum { TZ_SCALE_NONE = 0, TZ_SCALE_C_ROWS = 1, TZ_SCALE_S_COLS = 2 };
bool tsmm_oz_fits(int q, int nout);
bool launch_tsmm_oz(int64_t n, const Blocks3& S, const double* C, int ldc, int nx, int np, int w0p, double* out0,
                    double* out1, int64_t ldout, unsigned* status, unsigned skip, cudaStream_t st,
                    int scale_mode = TZ_SCALE_NONE, const int* sexp = nullptr);
// gramA (upper block triangle of the Gram blocks as printed, diagonal blocks symmetrised) and gramB from the
// summed partials.  If paper_lambda != null the X block of gramA is diag(lambda) and the
// diagonal blocks of gramB are identities (the Gram blocks as printed).
void launch_gram_finalize(int q, int nparts, const double* part, bool with_a, double* gramA,
                          double* gramB, const double* paper_lambda, const Blocks3* widths,
                          cudaStream_t st);

// Vout = Vin Rinv for b columns of type t (Rinv upper-triangular b x b, float64, column-major,
// device).  Vout may equal Vin (in place).  Skipped if *status & skip_mask.
void launch_apply_rinv(int64_t n, int b, DType t, void* Vin, int64_t ldin, void* Vout,
                       int64_t ldout, const double* Rinv, const unsigned* status,
                       unsigned skip_mask, cudaStream_t st);
// Ritz update (the update of X and P): Pout = S1 C1 + S2 C2 (type of S1, S2) and
// Xout = S0 C0 + Pout (float64), with C (q x m, column-major, ld q, float64) split by rows into
// C0 (w0), C1 (w1), C2 (w2).  Xout may alias S0 and Pout may alias S2; Pout may be null.
// Skipped if *status & skip_mask.
// If Xh is non-null, also writes the float32 hi / lo planes of Xout (mixed form).
void launch_update(int64_t n, int m, const Blocks3& S, const double* C, double* Xout,
                   void* Pout, int64_t ldout, const unsigned* status, unsigned skip_mask,
                   cudaStream_t st, float* Xh = nullptr, float* Xl = nullptr);

// Coefficients of the constraint projection V - Y (Y^T V) (the constraint projections with an orthonormal
// Y): C ((b + k) x b) = [I; -(Y^T V)] from the Gram matrix G of [V Y] ((b + k) x (b + k)), for
// launch_update over the blocks [V Y].
void launch_proj_coef(int b, int k, const double* G, double* C, cudaStream_t st);

// gramA / gramB of the residual form from its partial sums (nparts chunks of 2 q^2 doubles,
// q = m + b + bp; see launch_gram_mx2).
void launch_gram_finalize_mx(int q, int m, int b, int bp, int nparts, const double* part,
                             const double* lam, double* gramA, double* gramB, cudaStream_t st);
// ---------------------------------------------------------------- TMA-staged float32 Grams
// (k_gram32.cu).  Blocks are float32, 16-byte aligned, with a common leading dimension ld
// divisible by 4.  Partial sums go to `part` (g32_chunks(n) chunks; part_doubles is checked).
// A kernel whose bounded wait gives up sets ST_TIMEOUT in *status.
int g32_chunks(int64_t n);
// C = [S0 S1]^T V ((w0 + w1) x b, column-major, ld w0 + w1) and, if G != null, G = V^T V
// (b x b, symmetric), float64 chunk sums of per-chunk float32 sums.  tc (GramTc): whether the
// tensor cores (3 x TF32 products, k_gram_tc.cu) may run them, else float32 products with
// compensated sums on the SIMT pipes.
void launch_gram32_cross(int64_t n, int64_t ld, const float* S0, int w0, const float* S1, int w1,
                         const float* V, int b, double* C, double* G, double* part,
                         int64_t part_doubles, unsigned* status, int tc, cudaStream_t st);
// G -= C^T C (G b x b symmetric, C w x b column-major with leading dimension ldc), float64.
void launch_gram_sub_ctc(int w, int b, const double* C, int ldc, double* G, cudaStream_t st);
// Residual-form Gram of the mixed form, S = [X W P] (X as hi / lo planes Xh, Xl), T = [R AW AP]
// (R = AX - X Lambda): float32 products for every block but X^T X (engine as in
// launch_gram32_cross), double-float tiles for X^T X, then gramA, gramB
// (q x q, q = m + b + bp).
void launch_gram_mx2(int64_t n, int64_t ld, const float* Xh, const float* Xl, const float* W,
                     const float* P, const float* R, const float* AW, const float* AP, int m, int b,
                     int bp, double* part, int64_t part_doubles, const double* lam, double* gramA,
                     double* gramB, unsigned* status, int tc, cudaStream_t st);
// ---------------------------------------------------------------- mixed form, X as planes
// (k_mixed.cu).  X = Xh + Xl (float32 hi / lo planes, ld divisible by 4).
// R = A X - X diag(lam) (double-float stencil, R float32) for m columns, and per-block sums of
// squares: partial[j * resid_mx_blocks(g) + block] (add them with launch_norms_finalize).
int resid_mx_blocks(const Grid3& g);
void launch_resid_mx(const Grid3& g, int m, double scale, const float* Xh, const float* Xl,
                     int64_t ld, const double* lam, float* R, int64_t ldr, double* partial,
                     cudaStream_t st);
// X = Xh + Xl in float64.
void launch_planes_to_f64(int64_t n, int m, const float* Xh, const float* Xl, int64_t ld, double* X,
                          int64_t ldx, cudaStream_t st);
// ---------------------------------------------------------------- TMA-streamed float32 products
// (k_tsmm.cu).  Blocks float32, 16-byte aligned, ld divisible by 4; a kernel whose bounded wait
// gives up sets ST_TIMEOUT in *err.
// V <- V - [L0 L1] C for b columns of V (C (w0 + w1) x b, column-major, ld ldc, float64).
void launch_project32(int64_t n, int b, float* V, const float* L0, int w0, const float* L1, int w1,
                      int64_t ld, const double* C, int ldc, unsigned* err, cudaStream_t st);
// V <- [L0 L1 V] K (K (w0 + w1 + b) x b, column-major, ld ldk, float64), in place; skipped if
// *status & skip.  With K = [-C Rinv; Rinv] it is the last Gram-Schmidt pass and the Cholesky
// step in one pass over V.
void launch_combine32(int64_t n, int b, float* V, const float* L0, int w0, const float* L1, int w1, int64_t ld,
                      const double* K, int ldk, const unsigned* status, unsigned skip, unsigned* err,
                      cudaStream_t st);
// K = [-C Rinv; Rinv] ((w + b) x b, ld w + b) for C (w x b, ld ldc) and upper Rinv (b x b).
void launch_projapply_coef(int w, int b, const double* C, int ldc, const double* Rinv, double* K,
                           const unsigned* status, unsigned skip, cudaStream_t st);
// V <- V Rinv (Rinv b x b upper triangular, ld b, float64), in place; skipped if *status & skip.
void launch_apply32(int64_t n, int b, float* V, int64_t ld, const double* Rinv,
                    const unsigned* status, unsigned skip, unsigned* err, cudaStream_t st);
// Ritz update of the mixed form: Pout = W C_W + P C_P (float32) and X = X C_X + Pout in
// double-float with X = Xh + Xl (in place), C q x m column-major (ld q) with rows C_X (m), C_W (b),
// C_P (bp); Pout may alias P or be null.  Skipped if *status & skip.
void launch_update_mx2(int64_t n, int m, float* Xh, float* Xl, const float* W, int b, const float* P,
                       int bp, int64_t ld, const double* C, int q, float* Pout, const unsigned* status,
                       unsigned skip, unsigned* err, cudaStream_t st);
// ---------------------------------------------------------------- variable coefficients
// (k_varcoef.cu).  Face coefficients in the layout x-, y-, z-faces (x fastest), float64.
int64_t vc_num_faces(const Grid3& g);
// mode 0: y = A x;  1: y = (1-w) x + w (z/scale + N x)/D (Jacobi, e = x, r = z);
// 2: y = z - A x;  3: y = w z / (scale D)  -- A = scale (D - N), D = sum of the 6 faces.
void launch_vc_sweep(const Grid3& g, int mode, int ncols, const double* kap, double scale, double w,
                     const double* x, int64_t ldx, const double* z, int64_t ldz, double* y,
                     int64_t ldy, cudaStream_t st);
// Coarse-level faces (harmonic along the normal, 1/4-1/2-1/4 across, / 4).
void launch_vc_coarsen(const Grid3& gf, const Grid3& gc, const double* kf, double* kc, cudaStream_t st);
// Ainv = A^-1 of the operator on the (small) grid g via a dense Cholesky factor; A and work are
// n x n scratch; *fail set if A is not positive definite.
void launch_vc_coarse_inverse(const Grid3& g, const double* kap, double scale, double* A, double* work,
                              double* Ainv, int* fail, cudaStream_t st);
// e = Ainv r for ncols columns (Ainv n x n column-major).
void launch_dense_apply(int n, int ncols, const double* Ainv, const double* r, int64_t ldr, double* e,
                        int64_t lde, cudaStream_t st);
// grad[f] = scale sum_i w[i] (x_i,q - x_i,p)^2 (w host array of m weights).
void launch_vc_grad(const Grid3& g, int m, const double* w, double scale, const double* X, int64_t ldx,
                    double* grad, cudaStream_t st);
// ---------------------------------------------------------------- inner PCG (k_pcg.cu)
// b independent PCG solves, float64 columns with leading dimension ld.  Column dots u_j . v_j into
// out[j] via pcg_chunks(n) * b partial sums (fixed-order chunk sums); act[j] is cleared when
// out[j] <= 0 (act may not be null).
int pcg_chunks(int64_t n);
void launch_coldot(int64_t n, int b, const double* U, const double* V, int64_t ld, double* partial, double* out,
                   int* act, cudaStream_t st);
void launch_fill_int(int b, int v, int* a, cudaStream_t st);
// E += alpha P, R -= alpha AP, alpha_j = rz_j / pap_j, on columns with act[j].
void launch_pcg_er(int64_t n, int b, const double* rz, const double* pap, const int* act, double* E, double* R,
                   const double* P, const double* AP, int64_t ld, cudaStream_t st);
// P = Z + beta P, beta_j = rz_new_j / rz_j, on columns with act[j].
void launch_pcg_p(int64_t n, int b, const double* rz_new, const double* rz, const int* act, double* P,
                  const double* Z, int64_t ld, cudaStream_t st);

// ---------------------------------------------------------------- small dense
// Rinv = R^-1, R = chol(G) on the unit-diagonal scaling of G (b x b).  On failure sets
// fail_bit in *status and leaves Rinv unspecified.  Skipped if *status & skip_mask.
void launch_chol_rinv(int b, const double* G, double* Rinv, unsigned* status, unsigned fail_bit,
                      unsigned skip_mask, cudaStream_t st);
// Rayleigh-Ritz: gramA C = gramB C Lambda (q x q), m smallest.  q_min is the size without the
// P block (used if the full gramB is not positive definite: sets ST_P_DROPPED; if that
// fails too, sets ST_RR_BREAKDOWN).  lam (m), C (q x m, ld q; P rows zero when dropped).
// Skipped if *status & skip_mask.  `work` has rr_work_doubles(q) doubles.
int64_t rr_work_doubles(int q);
void launch_rayleigh_ritz(int q, int q_min, int m, const double* gramA, const double* gramB,
                          double* lam, double* C, double* work, unsigned* status,
                          unsigned skip_mask, cudaStream_t st);

}  // namespace lg
