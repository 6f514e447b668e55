// Small dense kernels of one LOBPCG iteration, in float64, each on one thread block:
//  * k_chol_rinv: the scale-invariant Cholesky factor of a b x b Gram matrix and its inverse
//    (Algorithm steps 3, 11, 14; the paper requires invariance to column scaling, Section 2.2,
//    so the factor is computed on D G D with D = diag(G)^-1/2 and R = R' D^-1).
//  * k_rayleigh_ritz: Algorithm step 24, gramA C = gramB C Lambda.  gramB is reduced by its
//    scaled Cholesky factor (B_s = D gramB D = L L^T), the standard problem
//    M = L^-1 (D gramA D) L^-T is diagonalised by the cyclic Jacobi method with the
//    round-robin parallel ordering (Golub & Van Loan, Matrix Computations, Sec. 8.5), and
//    C = D L^-T V holds gramB-orthonormal eigenvectors.
// Breakdown rule of both: a pivot of the unit-diagonal matrix at or below order * 2^-52 fails.
#include "common.cuh"

namespace lg {
namespace {

constexpr double kEps = 2.220446049250313e-16;   // 2^-52

// Lower-triangular inverse, column by column: warp w owns columns w, w + nwarps, ...; lane l
// owns rows l, l + 32, l + 64 of the column.  L and Linv are row-major with leading dim ldl.
__device__ void lower_inverse(int nq, const double* L, int ldl, double* Linv, int ldi) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < nq; j += nw) {
        double x[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) x[r] = (lane + 32 * r == j) ? 1.0 : 0.0;
        for (int k = j; k < nq; ++k) {
            const int ok = k & 31, rk = k >> 5;
            double xk = 0.0;
#pragma unroll
            for (int r = 0; r < 3; ++r)
                if (r == rk && lane == ok) { x[r] = x[r] / L[k * ldl + k]; xk = x[r]; }
            xk = __shfl_sync(0xffffffffu, xk, ok);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int i = lane + 32 * r;
                if (i > k && i < nq) x[r] = fma(-L[i * ldl + k], xk, x[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
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

__global__ void k_chol_rinv(int b, const double* __restrict__ G, double* __restrict__ Rinv,
                            unsigned* status, unsigned fail_bit, unsigned skip) {
    __shared__ double S[kMaxM * (kMaxM + 1)];
    __shared__ double Li[kMaxM * (kMaxM + 1)];
    __shared__ double d[kMaxM];
    __shared__ int flag;
    if (status && (*status & skip)) return;
    const int ld = kMaxM + 1;
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

// ------------------------------------------------------------------ Rayleigh-Ritz
constexpr int kRRThreads = 1024;

__global__ void __launch_bounds__(kRRThreads)
    k_rayleigh_ritz(int q, int q_min, int m, int b_identity, const double* __restrict__ gA,
                    const double* __restrict__ gB, double* __restrict__ lam,
                    double* __restrict__ C, double* __restrict__ work, unsigned* status,
                    unsigned skip) {
    extern __shared__ double sm[];
    const int ld = q + 1;
    double* M = sm;               // q x (q+1), row-major
    double* V = sm + q * ld;      // q x (q+1), row-major
    __shared__ double d[kMaxQ + 1];
    __shared__ double rc[kMaxQ / 2 + 1], rs[kMaxQ / 2 + 1];
    __shared__ int rp[kMaxQ / 2 + 1], rr[kMaxQ / 2 + 1];
    __shared__ int ord[kMaxQ + 1], perm[kMaxQ];
    __shared__ int flag, rotated;
    __shared__ double jthr;
    if (status && (*status & skip)) return;
    double* Linv = work;                       // q x q row-major (ld q)
    double* T1 = work + (int64_t)q * q;        // q x q row-major
    const int tid = threadIdx.x;

    // The P block is already out if chol(P_J^T P_J) failed this iteration (steps 13-16).
    int nq = (*status & ST_P_DROPPED) ? q_min : q;
    for (;;) {
        // ---- scaled Cholesky of gramB (leading nq x nq block), in V
        if (tid == 0) flag = 0;
        __syncthreads();
        for (int i = tid; i < nq; i += blockDim.x) {
            const double g = b_identity ? 1.0 : gB[i + (int64_t)q * i];
            if (!(g > 0.0) || !isfinite(g)) flag = 1;
            d[i] = 1.0 / sqrt(g);
        }
        __syncthreads();
        if (!flag) {
            for (int e = tid; e < nq * nq; e += blockDim.x) {
                const int i = e / nq, j = e % nq;
                const double g = b_identity ? (i == j ? 1.0 : 0.0) : gB[i + (int64_t)q * j];
                V[i * ld + j] = d[i] * g * d[j];
            }
            __syncthreads();
            cholesky_lower(nq, V, ld, &flag);
        }
        __syncthreads();
        if (!flag) break;
        if (nq > q_min) {
            nq = q_min;
            if (tid == 0) atomicOr(status, (unsigned)ST_P_DROPPED);
            __syncthreads();
            continue;
        }
        if (tid == 0) atomicOr(status, (unsigned)ST_RR_BREAKDOWN);
        return;
    }
    // ---- Linv = L^-1; T1 = Linv * (D gA D); M = T1 * Linv^T
    lower_inverse(nq, V, ld, Linv, q);
    __syncthreads();
    for (int e = tid; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s = fma(Linv[i * q + k], d[k] * gA[k + (int64_t)q * j], s);
        T1[i * q + j] = s * d[j];
    }
    __syncthreads();
    for (int e = tid; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        double s = 0.0;
        for (int k = 0; k <= j; ++k) s = fma(T1[i * q + k], Linv[j * q + k], s);
        M[i * ld + j] = s;
    }
    __syncthreads();
    // symmetrise (rounding) and V = I
    for (int e = tid; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        if (i < j) {
            const double a = 0.5 * (M[i * ld + j] + M[j * ld + i]);
            M[i * ld + j] = a;
            M[j * ld + i] = a;
        }
        V[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    // ---- cyclic Jacobi, round-robin ordering over qe = nq rounded up to even.  A pair is
    // rotated while |M_pr| > eps ||M||_F: the backward-stable threshold (a relative test against
    // sqrt(|M_pp M_rr|) would chase the eps ||M|| noise that every rotation leaves behind).
    const int qe = nq + (nq & 1);
    const int npairs = qe / 2;
    for (int i = tid; i < qe; i += blockDim.x) ord[i] = i;
    {
        double ss = 0.0;
        for (int e = tid; e < nq * nq; e += blockDim.x) {
            const double v = M[(e / nq) * ld + e % nq];
            ss = fma(v, v, ss);
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
        if ((tid & 31) == 0) rc[tid >> 5] = ss;   // rc is free until the sweeps start
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += rc[w];
            jthr = kEps * sqrt(t);
        }
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < qe - 1; ++step) {
            if (tid < npairs) {
                int p = ord[tid], r = ord[qe - 1 - tid];
                if (p > r) { const int t = p; p = r; r = t; }
                double c = 1.0, s = 0.0;
                if (r < nq) {
                    const double apq = M[p * ld + r], app = M[p * ld + p], arr = M[r * ld + r];
                    if (fabs(apq) > jthr) {
                        const double tau = (arr - app) / (2.0 * apq);
                        const double t = copysign(1.0, tau) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
                        c = 1.0 / sqrt(fma(t, t, 1.0));
                        s = t * c;
                        rotated = 1;
                    }
                }
                rc[tid] = c; rs[tid] = s; rp[tid] = p; rr[tid] = r;
            }
            __syncthreads();
            // rows: M <- J^T M
            for (int e = tid; e < npairs * nq; e += blockDim.x) {
                const int k = e / nq, j = e % nq;
                const double c = rc[k], s = rs[k];
                if (s == 0.0) continue;
                const int p = rp[k], r = rr[k];
                const double mp = M[p * ld + j], mr = M[r * ld + j];
                M[p * ld + j] = c * mp - s * mr;
                M[r * ld + j] = fma(s, mp, c * mr);
            }
            __syncthreads();
            // columns: M <- M J, V <- V J
            for (int e = tid; e < npairs * nq; e += blockDim.x) {
                const int k = e / nq, i = e % nq;
                const double c = rc[k], s = rs[k];
                if (s == 0.0) continue;
                const int p = rp[k], r = rr[k];
                const double mp = M[i * ld + p], mr = M[i * ld + r];
                M[i * ld + p] = c * mp - s * mr;
                M[i * ld + r] = fma(s, mp, c * mr);
                const double vp = V[i * ld + p], vr = V[i * ld + r];
                V[i * ld + p] = c * vp - s * vr;
                V[i * ld + r] = fma(s, vp, c * vr);
            }
            __syncthreads();
            if (tid < npairs && rs[tid] != 0.0) {
                M[rp[tid] * ld + rr[tid]] = 0.0;
                M[rr[tid] * ld + rp[tid]] = 0.0;
            }
            if (tid == 0) {   // rotate positions 1..qe-1 of the round-robin schedule
                const int last = ord[qe - 1];
                for (int i = qe - 1; i > 1; --i) ord[i] = ord[i - 1];
                ord[1] = last;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // ---- ascending order (stable), eigenvalues and C = D L^-T V
    for (int i = tid; i < nq; i += blockDim.x) {
        const double li = M[i * ld + i];
        int rank = 0;
        for (int j = 0; j < nq; ++j) {
            const double lj = M[j * ld + j];
            rank += (lj < li) || (lj == li && j < i);
        }
        perm[rank] = i;
        if (!isfinite(li)) atomicOr(status, (unsigned)ST_NONFINITE);
    }
    __syncthreads();
    for (int r = tid; r < m; r += blockDim.x) lam[r] = M[perm[r] * ld + perm[r]];
    for (int e = tid; e < q * m; e += blockDim.x) {
        const int i = e % q, r = e / q;
        double s = 0.0;
        if (i < nq) {
            const int pc = perm[r];
            for (int k = i; k < nq; ++k) s = fma(Linv[k * q + i], V[k * ld + pc], s);
            s *= d[i];
        }
        C[i + (int64_t)q * r] = s;
    }
}

}  // namespace

void launch_chol_rinv(int b, const double* G, double* Rinv, unsigned* status, unsigned fail_bit,
                      unsigned skip_mask, cudaStream_t st) {
    LG_REQUIRE(b >= 1 && b <= kMaxM, LOBPCG_ERR_ARG, "block width out of range");
    k_chol_rinv<<<1, 256, 0, st>>>(b, G, Rinv, status, fail_bit, skip_mask);
    LG_CHECK_LAUNCH();
}

int64_t rr_work_doubles(int q) { return 2 * (int64_t)q * q; }

void launch_rayleigh_ritz(int q, int q_min, int m, const double* gramA, const double* gramB,
                          double* lam, double* C, double* work, unsigned* status,
                          unsigned skip_mask, cudaStream_t st) {
    LG_REQUIRE(q >= 1 && q <= kMaxQ && m <= q && q_min >= m && q_min <= q, LOBPCG_ERR_ARG,
               "Rayleigh-Ritz size out of range");
    const size_t smem = 2 * (size_t)q * (q + 1) * sizeof(double);
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    static bool attr_set[64] = {false};
    if (dev < 64 && !attr_set[dev]) {
        LG_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * (size_t)kMaxQ * (kMaxQ + 1) * sizeof(double))));
        attr_set[dev] = true;
    }
    k_rayleigh_ritz<<<1, kRRThreads, smem, st>>>(q, q_min, m, gramB == nullptr ? 1 : 0, gramA,
                                                  gramB, lam, C, work, status, skip_mask);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
