// Small dense kernels of one LOBPCG iteration, in float64, each on one thread block:
//  * k_chol_rinv: the scale-invariant Cholesky factor of a b x b Gram matrix and its inverse
//    (Section 2.2; the paper requires invariance to column scaling, Section 2.2,
//    so the factor is computed on D G D with D = diag(G)^-1/2 and R = R' D^-1).
//  (the Rayleigh-Ritz step lives in k_rr.cu)
// Breakdown rule of both: a pivot of the unit-diagonal matrix at or below order * 2^-52 fails.
#include "common.cuh"

namespace lg {
namespace {

constexpr double kEps = 2.220446049250313e-16;   // 2^-52

constexpr int kRowsPerLane = (kMaxM + 31) / 32;

// Lower-triangular inverse, column by column: warp w owns columns w, w + nwarps, ...; lane l
// owns rows l, l + 32, l + 64, ... of the column.  L and Linv are row-major with leading dim ldl.
__device__ void lower_inverse(int nq, const double* L, int ldl, double* Linv, int ldi) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < nq; j += nw) {
        double x[kRowsPerLane];
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) x[r] = (lane + 32 * r == j) ? 1.0 : 0.0;
        for (int k = j; k < nq; ++k) {
            const int ok = k & 31, rk = k >> 5;
            double xk = 0.0;
#pragma unroll
            for (int r = 0; r < kRowsPerLane; ++r)
                if (r == rk && lane == ok) { x[r] = x[r] / L[k * ldl + k]; xk = x[r]; }
            xk = __shfl_sync(0xffffffffu, xk, ok);
#pragma unroll
            for (int r = 0; r < kRowsPerLane; ++r) {
                const int i = lane + 32 * r;
                if (i > k && i < nq) x[r] = fma(-L[i * ldl + k], xk, x[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) {
            const int i = lane + 32 * r;
            if (i < nq) Linv[i * ldi + j] = (i >= j) ? x[r] : 0.0;
        }
    }
}

// In-place right-looking Cholesky of the nq x nq row-major matrix S (lower triangle used).
// Returns false on a pivot <= nq * eps or a non-finite pivot.  Must be called by all threads.
__device__ bool cholesky_lower(int nq, double* S, int lds, int* flag) {
    for (int k = 0; k < nq; ++k) {
        if (threadIdx.x == 0) {
            const double piv = S[k * lds + k];
            if (!(piv > nq * kEps) || !isfinite(piv)) *flag = 1;
            else S[k * lds + k] = sqrt(piv);
        }
        __syncthreads();
        if (*flag) return false;
        const double lkk = S[k * lds + k];
        for (int i = k + 1 + threadIdx.x; i < nq; i += blockDim.x) S[i * lds + k] /= lkk;
        __syncthreads();
        const int rem = nq - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j <= i) S[i * lds + j] = fma(-S[i * lds + k], S[j * lds + k], S[i * lds + j]);
        }
        __syncthreads();
    }
    return true;
}

// S and its inverse Li (b x (b + 1) each, row-major) in dynamic shared memory.
__global__ void k_chol_rinv(int b, const double* __restrict__ G, double* __restrict__ Rinv,
                            unsigned* status, unsigned fail_bit, unsigned skip) {
    extern __shared__ double smd[];
    __shared__ double d[kMaxM];
    __shared__ int flag;
    if (status && (*status & skip)) return;
    const int ld = b + 1;
    double* S = smd;
    double* Li = smd + b * ld;
    if (threadIdx.x == 0) flag = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x)
        if (!isfinite(G[e])) {
            flag = 1;
            if (status) atomicOr(status, (unsigned)ST_NONFINITE);
        }
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
        const double g = G[i + (int64_t)b * i];
        if (!(g > 0.0) || !isfinite(g)) flag = 1;
        d[i] = 1.0 / sqrt(g);
    }
    __syncthreads();
    if (!flag) {
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int i = e % b, j = e / b;
            S[i * ld + j] = d[i] * G[e] * d[j];
        }
        __syncthreads();
        cholesky_lower(b, S, ld, &flag);
    }
    __syncthreads();
    if (flag) {
        if (threadIdx.x == 0 && status) atomicOr(status, fail_bit);
        return;
    }
    lower_inverse(b, S, ld, Li, ld);
    __syncthreads();
    // R^-1 = D L^-T:  Rinv[i][j] = d_i * Linv[j][i]  (upper triangular), column-major output.
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int i = e % b, j = e / b;
        Rinv[e] = (i <= j) ? d[i] * Li[j * ld + i] : 0.0;
    }
}

}  // namespace

void launch_chol_rinv(int b, const double* G, double* Rinv, unsigned* status, unsigned fail_bit,
                      unsigned skip_mask, cudaStream_t st) {
    LG_REQUIRE(b >= 1 && b <= kMaxM, LOBPCG_ERR_ARG, "block width out of range");
    const size_t smem = 2 * (size_t)b * (b + 1) * sizeof(double);
    static bool attr[64] = {};
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    if (smem > 48 * 1024 && dev < 64 && !attr[dev]) {
        LG_CUDA(cudaFuncSetAttribute((const void*)k_chol_rinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * (size_t)kMaxM * (kMaxM + 1) * sizeof(double))));
        attr[dev] = true;
    }
    k_chol_rinv<<<1, 256, smem, st>>>(b, G, Rinv, status, fail_bit, skip_mask);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
