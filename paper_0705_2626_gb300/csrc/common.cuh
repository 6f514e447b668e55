// Shared definitions of the GB300 LOBPCG library: error type, grid geometry,
// column lists and the host-side launchers of every kernel.  Kernels live in
// k_stencil.cu (stencil family + V-cycle), k_block.cu (tall-skinny block ops)
// and k_dense.cu (small dense factorizations on one thread block).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <stdexcept>
#include <string>

#include "../../include/lobpcg_gb300.h"

namespace lg {

extern std::atomic<long long> g_kernel_launches;

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
    ST_W_BREAKDOWN = 1u,      // chol(W_J^T W_J) failed (step 11)
    ST_P_DROPPED = 2u,        // P block dropped this iteration (chol of P or gramB failed)
    ST_RR_BREAKDOWN = 4u,     // gramB not positive definite without P
    ST_X_BREAKDOWN = 8u,      // chol(X^T X) failed (step 3)
    ST_NONFINITE = 16u,       // non-finite value in a small dense matrix
};

// ---------------------------------------------------------------- stencil family
// y = a*x + b*(sum of the 6 neighbours of x) [+ c*z], per column, zero outside the grid.
void launch_stencil_axpby(const Grid3& g, int ncols, double a, double b, const double* x,
                          int64_t ldx, double c, const double* z, int64_t ldz, double* y,
                          int64_t ldy, cudaStream_t st);
// Full-weighting restriction rc = P^T rf / 8 (fine grid gf -> coarse grid gc).
void launch_restrict(const Grid3& gf, const Grid3& gc, int ncols, const double* rf, int64_t ldf,
                     double* rc, int64_t ldc, cudaStream_t st);
// Trilinear prolongation with correction: ef += P ec.
void launch_prolong_add(const Grid3& gf, const Grid3& gc, int ncols, const double* ec,
                        int64_t ldc, double* ef, int64_t ldf, cudaStream_t st);
// Exact coarsest-level solve e = A_c^-1 r through the discrete sine transform.
// `tables` holds the three normalised 1-D sine matrices and the eigenvalues
// (layout from coarse_tables_size / launch_coarse_setup).
int64_t coarse_tables_size(const Grid3& g);
void launch_coarse_setup(const Grid3& g, double scale, double* tables, cudaStream_t st);
void launch_coarse_solve(const Grid3& g, int ncols, const double* tables, const double* r,
                         int64_t ldr, double* e, int64_t lde, cudaStream_t st);

// ---------------------------------------------------------------- block ops
void launch_random_block(uint64_t seed, int64_t n, int m, double* X, int64_t ldx,
                         cudaStream_t st);
// Partial sums of squares of W[:, t] = AX[:, cols[t]] - lambda[cols[t]] * X[:, cols[t]];
// writes W if non-null.  partial has nchunks * cols.n doubles.
int residual_chunks(int64_t n);
void launch_residual(int64_t n, const ColList& cols, const double* X, const double* AX,
                     int64_t ld, const double* lambda, double* W, int64_t ldw, double* partial,
                     cudaStream_t st);
// norms[t] = sqrt(sum_c partial[t*nchunks + c]) in a fixed order.
void launch_norms_finalize(int ncols, int nchunks, const double* partial, double* norms,
                           cudaStream_t st);

// Block pointers of a basis [B0 B1 B2] (widths w[k], common leading dimension).
struct Blocks3 {
    const double* p[3];
    int w[3];
    int64_t ld;
    __host__ __device__ int q() const { return w[0] + w[1] + w[2]; }
};
// Gram partial sums over `nparts` row ranges: part has nparts * 2*q*q doubles.
int gram_parts(int64_t n);
int64_t gram_scratch_doubles(int64_t n, int q);
void launch_gram(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int nparts,
                 cudaStream_t st);
// gramA = (G + G^T)/2 of the summed A partials; gramB = summed B partials, mirrored.
// If paper_lambda != null the X block of gramA is diag(lambda) and the diagonal blocks of
// gramB are identities (steps 18-22 as printed).
void launch_gram_finalize(int q, int nparts, const double* part, bool with_a, double* gramA,
                          double* gramB, const double* paper_lambda, const Blocks3* widths,
                          cudaStream_t st);

// Vout = Vin Rinv for b columns (Rinv upper-triangular b x b, column-major, device).
// Vout may equal Vin (in place).  Skipped if *status & skip_mask.
void launch_apply_rinv(int64_t n, int b, const double* Vin, int64_t ldin, double* Vout,
                       int64_t ldout, const double* Rinv, const unsigned* status,
                       unsigned skip_mask, cudaStream_t st);
// Ritz update (steps 27-28 / 31-32): Pout = S1 C1 + S2 C2 and Xout = S0 C0 + Pout, with
// C (q x m, column-major, ld q) split by rows into C0 (w0), C1 (w1), C2 (w2).
// Xout may alias S0 and Pout may alias S2.  Skipped if *status & skip_mask.
void launch_update(int64_t n, int m, const Blocks3& S, const double* C, double* Xout,
                   double* Pout, int64_t ldout, const unsigned* status, unsigned skip_mask,
                   cudaStream_t st);

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
