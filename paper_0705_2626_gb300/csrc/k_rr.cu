// Rayleigh-Ritz step (Section 2.2): gramA C = gramB C Lambda, the m smallest eigenpairs,
// C gramB-orthonormal.  GB300 runs float64 at 1/64 of the float32 rate, and one thread block
// alone would spend most of an iteration on the O(q^3) float64 work of a Jacobi eigensolver, so
// the work is split:
//   1. one block:  D = diag(gramB)^-1/2, L = chol(D gramB D) (dropping the P block if this fails),
//                  Linv = L^-1;
//   2. q blocks:   M = Linv (D gramA D) Linv^T, one column per block (float64);
//   3. one block:  cyclic Jacobi on M in float32 (round-robin parallel ordering, Golub & Van
//                  Loan Sec. 8.5) -> approximate eigenvectors V (orthogonal to ~1e-7);
//   4. q blocks:   two refinement steps of Ogita & Aishima ("Iterative refinement for symmetric
//                  eigenvalue decomposition", 2018), float64 matrix products only:
//                  R = I - V^T V, S = V^T M V, l_i = s_ii / (1 - r_ii),
//                  E_ij = (s_ij + l_j r_ij) / (l_j - l_i) for separated pairs whose correction
//                  is small (|E_ij| <= 1e-4), r_ij / 2 otherwise, V <- V + V E (each step
//                  squares the error of the refined pairs);
//      then one orthonormalisation step V <- V (I + (I - V^T V) / 2);
//   5. one block:  S = V^T M V is diagonal up to rounding except inside near-degenerate clusters;
//                  float64 cyclic Jacobi sweeps that rotate only the pairs above 8 eps ||S||_F
//                  finish it (rotations Q), eigenvalue order;
//   6. m blocks:   C = D Linv^T V Q for the m smallest, ascending, one column per block.
// The single-block kernels keep their matrices in shared memory while they fit (q up to about
// 100 in float64, 158 in float32) and in the global work area beyond that (q up to 300).
// Breakdown rule as elsewhere: a pivot of the unit-diagonal matrix at or below order * 2^-52.
#include <algorithm>

#include "common.cuh"

namespace lg {
namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int kSubMax = 48;    // largest cleanup submatrix kept beside S and Q in shared memory
constexpr size_t kRRSmemMax = 200 * 1024;   // dynamic shared memory of the single-block kernels
constexpr int kRowsPerLane = (kMaxQ + 31) / 32;

// work layout (doubles), all q x q matrices column-major with leading dimension q, except the
// row-major scratch copies noted at their kernels
struct RRWork {
    double *Linv, *M, *V, *V2, *MV, *S, *R, *E, *d, *hdr, *perm;   // hdr[0] = nq, hdr[1] = ||M||_F
    __host__ __device__ RRWork(double* w, int q) {
        const size_t q2 = (size_t)q * q;
        Linv = w; M = w + q2; V = w + 2 * q2; V2 = w + 3 * q2; MV = w + 4 * q2; S = w + 5 * q2;
        R = w + 6 * q2; E = w + 7 * q2; d = w + 8 * q2; hdr = d + q; perm = hdr + 8;
    }
};

// Shared memory of the single-block kernels for basis width q (0: the work area is used).
__host__ __device__ inline size_t rr_chol_smem(int q) {
    const size_t b = 2 * (size_t)q * (q + 1) * sizeof(double);
    return b <= kRRSmemMax ? b : 0;
}
__host__ __device__ inline size_t rr_jacobi_smem(int q) {
    const size_t b = 2 * (size_t)q * (q + 1) * sizeof(float);
    return b <= kRRSmemMax ? b : 0;
}
__host__ __device__ inline size_t rr_final_sub_bytes(int q) {
    const int s = q < kSubMax ? q : kSubMax;
    return 2 * (size_t)s * (s + 1) * sizeof(double);
}
__host__ __device__ inline bool rr_final_in_smem(int q) {
    return 2 * (size_t)q * (q + 1) * sizeof(double) + rr_final_sub_bytes(q) <= kRRSmemMax;
}
__host__ __device__ inline size_t rr_final_smem(int q) {
    return rr_final_in_smem(q) ? 2 * (size_t)q * (q + 1) * sizeof(double) + rr_final_sub_bytes(q)
                               : rr_final_sub_bytes(q);
}

__device__ __forceinline__ int nq_of(const RRWork& w) { return (int)w.hdr[0]; }

// ---------------------------------------------------------------- 1. Cholesky of gramB
__device__ bool chol_lower_rm(int nq, double* S, int lds, int* flag, double* rinv) {   // row-major, in place
    for (int k = 0; k < nq; ++k) {
        if (threadIdx.x == 0) {
            const double piv = S[k * lds + k];
            if (!(piv > nq * kEps) || !isfinite(piv)) {
                *flag = 1;
            } else {
                const double l = sqrt(piv);
                S[k * lds + k] = l;
                *rinv = 1.0 / l;    // one division per pivot; the column is scaled by multiplication
            }
        }
        __syncthreads();
        if (*flag) return false;
        const double inv = *rinv;
        for (int i = k + 1 + threadIdx.x; i < nq; i += blockDim.x) S[i * lds + k] *= inv;
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

// Linv (row-major) by column-parallel forward substitution: warp w owns columns w, w + nwarps,
// ...; lane l owns rows l, l + 32, l + 64, ...
__device__ void lower_inv(int nq, const double* L, int ldl, double* Li, int ldi, double* dinv) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) dinv[k] = 1.0 / L[k * ldl + k];
    __syncthreads();
    for (int j = wid; j < nq; j += nw) {
        double x[kRowsPerLane];
#pragma unroll
        for (int r = 0; r < kRowsPerLane; ++r) x[r] = (lane + 32 * r == j) ? 1.0 : 0.0;
        for (int k = j; k < nq; ++k) {
            const int ok = k & 31, rk = k >> 5;
            double xk = 0.0;
#pragma unroll
            for (int r = 0; r < kRowsPerLane; ++r)
                if (r == rk && lane == ok) { x[r] = x[r] * dinv[k]; xk = x[r]; }
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
            if (i < nq) Li[i * ldi + j] = (i >= j) ? x[r] : 0.0;
        }
    }
}

__global__ void __launch_bounds__(1024)
    k_rr_chol(int q, int q_min, int b_identity, const double* __restrict__ gB, double* work,
              unsigned* status, unsigned skip) {
    extern __shared__ double sm[];
    __shared__ int flag;
    __shared__ double rinv, dinv[kMaxQ];
    if (*status & skip) return;
    RRWork w(work, q);
    // L and its inverse, row-major: in shared memory (leading dimension q + 1) while they fit,
    // else in the work area's R and E (leading dimension q; both are free until the initial Rayleigh-Ritz step)
    const bool in_smem = rr_chol_smem(q) != 0;
    const int ld = in_smem ? q + 1 : q;
    double* Lsm = in_smem ? sm : w.R;
    double* Lism = in_smem ? sm + q * ld : w.E;
    int nq = (*status & ST_P_DROPPED) ? q_min : q;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) flag = 0;
        __syncthreads();
        for (int i = tid; i < nq; i += blockDim.x) {
            const double g = b_identity ? 1.0 : gB[i + (int64_t)q * i];
            if (!(g > 0.0) || !isfinite(g)) flag = 1;
            w.d[i] = 1.0 / sqrt(g);
        }
        __syncthreads();
        if (!flag) {
            for (int e = tid; e < nq * nq; e += blockDim.x) {
                const int i = e / nq, j = e % nq;
                const double g = b_identity ? (i == j ? 1.0 : 0.0) : gB[i + (int64_t)q * j];
                Lsm[i * ld + j] = w.d[i] * g * w.d[j];
            }
            __syncthreads();
            chol_lower_rm(nq, Lsm, ld, &flag, &rinv);
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
    lower_inv(nq, Lsm, ld, Lism, ld, dinv);
    __syncthreads();
    for (int e = tid; e < q * q; e += blockDim.x) {    // Linv column-major, zero outside nq
        const int i = e % q, j = e / q;
        w.Linv[e] = (i < nq && j < nq) ? Lism[i * ld + j] : 0.0;
    }
    if (tid == 0) w.hdr[0] = nq;
}

// ---------------------------------------------------------------- 2. M = Linv (D A D) Linv^T
// Block j: y = (D A D) l_j with l_j = row j of Linv, then M[:, j] = Linv y.
__global__ void k_rr_form_m(int q, const double* __restrict__ gA, double* work, const unsigned* status,
                            unsigned skip) {
    __shared__ double y[kMaxQ], l[kMaxQ];
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    const int j = blockIdx.x;
    if (j >= nq) return;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) l[k] = w.Linv[j + (int64_t)q * k] * w.d[k];
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k <= j; ++k) s = fma(gA[i + (int64_t)q * k], l[k], s);
        y[i] = s * w.d[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s = fma(w.Linv[i + (int64_t)q * k], y[k], s);
        w.M[i + (int64_t)q * j] = s;
    }
}

// ---------------------------------------------------------------- Jacobi sweeps (shared code)
// Cyclic Jacobi on the nq x nq symmetric matrix A (row-major, leading dim lda, in shared
// memory) accumulating the rotations into V (row-major, ldv).  Parallel ordering: the circle
// method of round-robin tournaments (Golub & Van Loan Sec. 8.5): in round t the index sets
// {pos(k, t), pos(qe-1-k, t)} with pos(0, t) = 0 and pos(i, t) = 1 + (i - 1 + t) mod (qe - 1)
// are disjoint pairs, and over qe - 1 rounds every pair meets once.  A pair is rotated while
// |A_pr| > thr.  Because the pairs of a round are disjoint, J^T A J splits into independent
// 2 x 2 blocks (pair k rows, pair l columns), so a round is: rotation parameters (one thread
// per pair), barrier, every 2 x 2 block and every row of V updated in place, barrier.
// Returns after a sweep without rotations or after max_sweeps.
__device__ __forceinline__ int rr_pos(int i, int t, int qe) { return i == 0 ? 0 : 1 + (i - 1 + t) % (qe - 1); }

template <typename T>
__device__ void jacobi_sweeps(int nq, T* A, int lda, T* V, int ldv, T thr, int max_sweeps, T* rc, T* rs,
                              int* rp, int* rr, int* rotated) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int qe = nq + (nq & 1);
    const int np = qe / 2;
    if (qe < 2) return;
    // *rotated holds 1 + the last sweep that rotated (no reset between barriers needed)
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int t = 0; t < qe - 1; ++t) {
            if (tid < np) {
                int p = rr_pos(tid, t, qe), r = rr_pos(qe - 1 - tid, t, qe);
                if (p > r) { const int x = p; p = r; r = x; }
                T c = 1, s = 0;
                if (r < nq) {
                    const T apq = A[p * lda + r];
                    if (fabs(apq) > thr) {
                        const T app = A[p * lda + p], arr = A[r * lda + r];
                        const T tau = (arr - app) / (T(2) * apq);
                        const T tt = copysign(T(1), tau) / (fabs(tau) + sqrt(fma(tau, tau, T(1))));
                        c = T(1) / sqrt(fma(tt, tt, T(1)));
                        s = tt * c;
                        *rotated = sweep + 1;
                    }
                }
                rc[tid] = c; rs[tid] = s; rp[tid] = p; rr[tid] = r;
            }
            __syncthreads();
            // 2 x 2 blocks (pair k rows, pair l columns): rows then columns rotated
            for (int k = wid; k < np; k += nw) {
                const T ck = rc[k], sk = rs[k];
                const int pk = rp[k], rk = rr[k];
                const bool vk = rk < nq;
                for (int l = lane; l < np; l += 32) {
                    const T sl = rs[l];
                    if (sk == T(0) && sl == T(0)) continue;
                    const T cl = rc[l];
                    const int pl = rp[l], rl = rr[l];
                    const bool vl = rl < nq;
                    const T a = A[pk * lda + pl];
                    const T b = vl ? A[pk * lda + rl] : T(0);
                    const T c0 = vk ? A[rk * lda + pl] : T(0);
                    const T d = (vk && vl) ? A[rk * lda + rl] : T(0);
                    const T a1 = ck * a - sk * c0, b1 = ck * b - sk * d;
                    const T c1 = fma(sk, a, ck * c0), d1 = fma(sk, b, ck * d);
                    T a2 = cl * a1 - sl * b1, b2 = fma(sl, a1, cl * b1);
                    T c2 = cl * c1 - sl * d1;
                    const T d2 = fma(sl, c1, cl * d1);
                    if (k == l && sk != T(0)) { b2 = T(0); c2 = T(0); }   // the annihilated pair
                    A[pk * lda + pl] = a2;
                    if (vl) A[pk * lda + rl] = b2;
                    if (vk) A[rk * lda + pl] = c2;
                    if (vk && vl) A[rk * lda + rl] = d2;
                }
            }
            // V <- V J: pair k columns of every row
            for (int k = wid; k < np; k += nw) {
                const T sk = rs[k];
                if (sk == T(0)) continue;
                const T ck = rc[k];
                const int pk = rp[k], rk = rr[k];
                for (int i = lane; i < nq; i += 32) {
                    const T vp = V[i * ldv + pk], vr = V[i * ldv + rk];
                    V[i * ldv + pk] = ck * vp - sk * vr;
                    V[i * ldv + rk] = fma(sk, vp, ck * vr);
                }
            }
            __syncthreads();
        }
        // every thread reads the flag before any thread can start the next sweep and write it
        const bool again = (*rotated == sweep + 1);
        __syncthreads();
        if (!again) break;
    }
}

template <typename T>
__device__ T frob_norm_sq(int nq, const T* A, int lda, T* red) {   // block reduction, all threads
    T ss = 0;
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const T v = A[(e / nq) * lda + e % nq];
        ss = fma(v, v, ss);
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    T t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------- 3. float32 Jacobi
__global__ void __launch_bounds__(1024)
    k_rr_jacobi32(int q, double* work, const unsigned* status, unsigned skip) {
    extern __shared__ float smf[];
    __shared__ float rc[kMaxQ / 2 + 1], rs[kMaxQ / 2 + 1], red[32];
    __shared__ int rp[kMaxQ / 2 + 1], rr[kMaxQ / 2 + 1], rotated;
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    // A and V in shared memory while they fit, else (float32, leading dimension nq) in the work
    // area's MV, which is free until the initial Rayleigh-Ritz step
    const bool in_smem = rr_jacobi_smem(q) != 0;
    const int ld = in_smem ? nq + 1 : nq;
    float* A = in_smem ? smf : reinterpret_cast<float*>(w.MV);
    float* V = A + nq * ld;
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        A[i * ld + j] = (float)(0.5 * (w.M[i + (int64_t)q * j] + w.M[j + (int64_t)q * i]));
        V[i * ld + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    const float nrm2 = frob_norm_sq<float>(nq, A, ld, red);
    if (threadIdx.x == 0) w.hdr[1] = 0.0;
    // 8 eps32 ||M||_F: below the float32 rounding noise that every rotation leaves behind
    jacobi_sweeps<float>(nq, A, ld, V, ld, 8.f * 1.2e-7f * sqrtf(nrm2), 12, rc, rs, rp, rr, &rotated);
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int i = e % q, j = e / q;
        w.V[e] = (i < nq && j < nq) ? (double)V[i * ld + j] : 0.0;
    }
}

// ---------------------------------------------------------------- 4. refinement products
// mode 0: MV[:, j] = M V[:, j].   mode 1: S[:, j] = V^T MV[:, j] and R[:, j] = e_j - V^T V[:, j].
// mode 2: S[:, j] = V^T MV[:, j] only.   mode 3: V2[:, j] = V[:, j] + V E[:, j].
// mode 4: R[:, j] = e_j - V^T V[:, j] only.   mode 5: V2[:, j] = V[:, j] + V R[:, j] / 2.
__global__ void k_rr_gemm(int q, int mode, double* work, const unsigned* status, unsigned skip) {
    __shared__ double x[kMaxQ], z[kMaxQ];
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    const int j = blockIdx.x;
    if (j >= nq) return;
    const double* B = (mode == 0 || mode == 4) ? w.V : (mode == 3 ? w.E : (mode == 5 ? w.R : w.MV));
    const double sc = mode == 5 ? 0.5 : 1.0;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        x[k] = sc * B[k + (int64_t)q * j];
        if (mode == 1) z[k] = w.V[k + (int64_t)q * j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        if (mode == 0 || mode == 3 || mode == 5) {          // (M or V) times x
            const double* A = mode == 0 ? w.M : w.V;
            double s = 0.0;
            for (int k = 0; k < nq; ++k) s = fma(A[i + (int64_t)q * k], x[k], s);
            if (mode == 0) w.MV[i + (int64_t)q * j] = s;
            else w.V2[i + (int64_t)q * j] = w.V[i + (int64_t)q * j] + s;
        } else if (mode == 4) {                             // e_j - V^T v_j
            double r = 0.0;
            for (int k = 0; k < nq; ++k) r = fma(w.V[k + (int64_t)q * i], x[k], r);
            w.R[i + (int64_t)q * j] = (i == j ? 1.0 : 0.0) - r;
        } else {                                            // V^T x (and V^T z)
            double s = 0.0, r = 0.0;
            for (int k = 0; k < nq; ++k) {
                const double v = w.V[k + (int64_t)q * i];
                s = fma(v, x[k], s);
                if (mode == 1) r = fma(v, z[k], r);
            }
            w.S[i + (int64_t)q * j] = s;
            if (mode == 1) w.R[i + (int64_t)q * j] = (i == j ? 1.0 : 0.0) - r;
        }
    }
}

// E of one refinement step: block j writes column j (every block recomputes the norms).
__global__ void __launch_bounds__(256) k_rr_oa_e(int q, double* work, const unsigned* status, unsigned skip) {
    __shared__ double lt[kMaxQ];
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    const int jcol = blockIdx.x;
    if (jcol >= nq) return;
    for (int i = threadIdx.x; i < nq; i += blockDim.x)
        lt[i] = w.S[i + (int64_t)q * i] / (1.0 - w.R[i + (int64_t)q * i]);
    __syncthreads();
    // delta = 2 (||S - diag(l)||_F + ||M||_F ||R||_F): Frobenius norms bound the 2-norms
    double a = 0.0, b = 0.0, c = 0.0;
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const int i = e % nq, j = e / nq;
        const double s = w.S[i + (int64_t)q * j] - (i == j ? lt[i] : 0.0);
        const double r = w.R[i + (int64_t)q * j];
        const double mm = w.M[i + (int64_t)q * j];
        a = fma(s, s, a); b = fma(r, r, b); c = fma(mm, mm, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    __shared__ double ra[32], rb[32], rcc[32];
    if ((threadIdx.x & 31) == 0) { ra[threadIdx.x >> 5] = a; rb[threadIdx.x >> 5] = b; rcc[threadIdx.x >> 5] = c; }
    __syncthreads();
    double sa = 0.0, sb = 0.0, sc = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { sa += ra[i]; sb += rb[i]; sc += rcc[i]; }
    const double delta = 2.0 * (sqrt(sa) + sqrt(sc) * sqrt(sb));
    // A pair is refined by the first-order formula only when it is separated (gap > delta) and
    // the correction is small both ways (|s_ij + l_j r_ij| <= 1e-4 |gap|, and likewise for ji),
    // so that the next step squares its error; E_ij + E_ji = r_ij keeps V orthonormalising.
    // Other pairs are only orthonormalised (r_ij / 2) and finished by the cleanup sweeps.
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        const int j = jcol;
        const double r = w.R[i + (int64_t)q * j];
        double ev = 0.5 * r;
        if (i != j) {
            const double gap = lt[j] - lt[i];
            const double nij = w.S[i + (int64_t)q * j] + lt[j] * r;
            const double nji = w.S[j + (int64_t)q * i] + lt[i] * w.R[j + (int64_t)q * i];
            if (fabs(gap) > delta && fabs(nij) <= 1e-4 * fabs(gap) && fabs(nji) <= 1e-4 * fabs(gap))
                ev = nij / gap;
        }
        w.E[i + (int64_t)q * j] = ev;
    }
}

// ---------------------------------------------------------------- 5. cleanup
// S symmetrised (A) and the cleanup rotations Q: in shared memory (row-major, leading dimension
// nq + 1) while they fit, else in the work area's R and E (row-major, leading dimension q).
// Writes Q row-major into E (leading dimension q), the order of the eigenvalues into perm and the
// m smallest eigenvalues into lam.
__global__ void __launch_bounds__(1024)
    k_rr_final(int q, int m, double* work, double* __restrict__ lam, unsigned* status, unsigned skip) {
    extern __shared__ double sm[];
    __shared__ double rc[kMaxQ / 2 + 1], rs[kMaxQ / 2 + 1], red[32], lsort[kMaxQ];
    __shared__ int rp[kMaxQ / 2 + 1], rr[kMaxQ / 2 + 1], rotated, act[kMaxQ], idx[kMaxQ], nact;
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    const bool in_smem = rr_final_in_smem(q);
    const int ld = in_smem ? nq + 1 : q;
    double* A = in_smem ? sm : w.R;               // S, symmetrised, row-major
    double* Q = in_smem ? sm + nq * ld : w.E;     // accumulated cleanup rotations, row-major
    double* sub = in_smem ? Q + nq * ld : sm;     // the cleanup submatrix and its rotations
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        A[i * ld + j] = 0.5 * (w.S[i + (int64_t)q * j] + w.S[j + (int64_t)q * i]);
        Q[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const double nrm2 = frob_norm_sq<double>(nq, A, ld, red);
    const double thr = 8.0 * kEps * sqrt(nrm2);
    // After the refinement only the pairs inside near-degenerate clusters stay above thr; the
    // cleanup runs on the submatrix of those indices (their couplings to the rest are below thr,
    // so leaving them out changes eigenvalues and vectors only at the rounding level).
    for (int i = threadIdx.x; i < nq; i += blockDim.x) act[i] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
        const int i = e / nq, j = e % nq;
        if (i != j && fabs(A[i * ld + j]) > thr) act[i] = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int na = 0;
        for (int i = 0; i < nq; ++i)
            if (act[i]) idx[na++] = i;
        nact = na;
    }
    __syncthreads();
    const int na = nact;
    if (na > kSubMax) {
        // many unresolved pairs (the refinement did not converge): sweep the whole matrix
        jacobi_sweeps<double>(nq, A, ld, Q, ld, thr, 16, rc, rs, rp, rr, &rotated);
    } else if (na >= 2) {
        const int lds = na + 1;
        double* As = sub;                  // na x na submatrix and its rotations
        double* Qs = As + na * lds;
        for (int e = threadIdx.x; e < na * na; e += blockDim.x) {
            const int a = e / na, b = e % na;
            As[a * lds + b] = A[idx[a] * ld + idx[b]];
            Qs[a * lds + b] = (a == b) ? 1.0 : 0.0;
        }
        __syncthreads();
        jacobi_sweeps<double>(na, As, lds, Qs, lds, thr, 16, rc, rs, rp, rr, &rotated);
        __syncthreads();
        for (int e = threadIdx.x; e < na * na; e += blockDim.x) {
            const int a = e / na, b = e % na;
            Q[idx[a] * ld + idx[b]] = Qs[a * lds + b];
            if (a == b) A[idx[a] * ld + idx[a]] = As[a * lds + a];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        const double li = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < nq; ++j) {
            const double lj = A[j * ld + j];
            rank += (lj < li) || (lj == li && j < i);
        }
        w.perm[rank] = (double)i;
        lsort[rank] = li;
        if (!isfinite(li)) atomicOr(status, (unsigned)ST_NONFINITE);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) lam[r] = lsort[r];
    if (in_smem)
        for (int e = threadIdx.x; e < nq * nq; e += blockDim.x) {
            const int i = e / nq, j = e % nq;
            w.E[i * (int64_t)q + j] = Q[i * ld + j];
        }
}

// ---------------------------------------------------------------- 6. output, one column per block
// y = V2 Q[:, perm r] (V2 the refined eigenvectors of M), then C[:, r] = D Linv^T y.
__global__ void __launch_bounds__(256)
    k_rr_out(int q, double* work, double* __restrict__ C, const unsigned* status, unsigned skip) {
    __shared__ double qc[kMaxQ], y[kMaxQ];
    if (*status & skip) return;
    RRWork w(work, q);
    const int nq = nq_of(w);
    const int r = blockIdx.x;
    const int pc = (int)w.perm[r];
    for (int k = threadIdx.x; k < nq; k += blockDim.x) qc[k] = w.E[k * (int64_t)q + pc];
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nq; ++k) s = fma(w.V2[i + (int64_t)q * k], qc[k], s);
        y[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q; i += blockDim.x) {
        double s = 0.0;
        if (i < nq) {
            for (int k = i; k < nq; ++k) s = fma(w.Linv[k + (int64_t)q * i], y[k], s);
            s *= w.d[i];
        }
        C[i + (int64_t)q * r] = s;
    }
}

void set_smem(const void* f, size_t bytes) {
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    LG_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

int64_t rr_work_doubles(int q) { return 8 * (int64_t)q * q + 3 * q + 8; }

void launch_rayleigh_ritz(int q, int q_min, int m, const double* gramA, const double* gramB,
                          double* lam, double* C, double* work, unsigned* status,
                          unsigned skip_mask, cudaStream_t st) {
    LG_REQUIRE(q >= 1 && q <= kMaxQ && m <= q && q_min >= m && q_min <= q, LOBPCG_ERR_ARG,
               "Rayleigh-Ritz size out of range");
    LG_REQUIRE(status != nullptr, LOBPCG_ERR_ARG, "Rayleigh-Ritz needs a status word");
    static bool attr[64] = {};
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr[dev]) {
        set_smem((const void*)k_rr_chol, kRRSmemMax);
        set_smem((const void*)k_rr_final, kRRSmemMax);
        set_smem((const void*)k_rr_jacobi32, kRRSmemMax);
        attr[dev] = true;
    }
    const unsigned skip = skip_mask | ST_RR_BREAKDOWN;
    k_rr_chol<<<1, 1024, rr_chol_smem(q), st>>>(q, q_min, gramB == nullptr ? 1 : 0, gramB, work, status, skip_mask);
    LG_CHECK_LAUNCH();
    k_rr_form_m<<<q, 128, 0, st>>>(q, gramA, work, status, skip);
    LG_CHECK_LAUNCH();
    k_rr_jacobi32<<<1, 1024, rr_jacobi_smem(q), st>>>(q, work, status, skip);
    LG_CHECK_LAUNCH();
    for (int it = 0; it < 2; ++it) {
        k_rr_gemm<<<q, 128, 0, st>>>(q, 0, work, status, skip);   // MV = M V
        LG_CHECK_LAUNCH();
        k_rr_gemm<<<q, 128, 0, st>>>(q, 1, work, status, skip);   // S, R
        LG_CHECK_LAUNCH();
        k_rr_oa_e<<<q, 256, 0, st>>>(q, work, status, skip);
        LG_CHECK_LAUNCH();
        k_rr_gemm<<<q, 128, 0, st>>>(q, 3, work, status, skip);   // V2 = V + V E
        LG_CHECK_LAUNCH();
        LG_CUDA(cudaMemcpyAsync(work + 2 * (size_t)q * q, work + 3 * (size_t)q * q,
                                (size_t)q * q * sizeof(double), cudaMemcpyDeviceToDevice, st));   // V = V2
    }
    // one more orthonormalisation step, V <- V (I + R / 2): the refinement steps leave V
    // orthonormal only to the square of their largest correction, and S below must be an exact
    // similarity transform of M for the cleanup to give eigenvectors of M
    k_rr_gemm<<<q, 128, 0, st>>>(q, 4, work, status, skip);       // R = I - V^T V
    LG_CHECK_LAUNCH();
    k_rr_gemm<<<q, 128, 0, st>>>(q, 5, work, status, skip);       // V2 = V + V R / 2
    LG_CHECK_LAUNCH();
    LG_CUDA(cudaMemcpyAsync(work + 2 * (size_t)q * q, work + 3 * (size_t)q * q, (size_t)q * q * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));    // V = V2
    k_rr_gemm<<<q, 128, 0, st>>>(q, 0, work, status, skip);       // MV = M V
    LG_CHECK_LAUNCH();
    k_rr_gemm<<<q, 128, 0, st>>>(q, 2, work, status, skip);       // S = V^T M V
    LG_CHECK_LAUNCH();
    k_rr_final<<<1, 1024, rr_final_smem(q), st>>>(q, m, work, lam, status, skip);
    LG_CHECK_LAUNCH();
    k_rr_out<<<m, 256, 0, st>>>(q, work, C, status, skip);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
