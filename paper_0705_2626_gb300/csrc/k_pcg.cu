// Inner preconditioned conjugate gradients as the LOBPCG preconditioner (the paper's Section
// 4.2, "Performance Versus the Number of Inner Iterations"): block kernels for b independent PCG
// solves A e_j = r_j, one per column, with their scalars kept on the device.
//
// Per iteration (float64, textbook recurrences): alpha_j = (r_j . z_j) / (p_j . A p_j),
// e_j += alpha_j p_j, r_j -= alpha_j A p_j, z_j = M r_j, beta_j = (r_j . z_j)_new / (r_j . z_j),
// p_j = z_j + beta_j p_j.  A column stops for good (alpha = beta = 0, so e, r and p stay put) once
// p . A p <= 0 or r . z <= 0; `act` carries that flag.  Column dot products are summed per chunk
// of rows and the chunks added in a fixed order, so results are deterministic.
#include <algorithm>

#include "common.cuh"

namespace lg {
namespace {

constexpr int kDotThreads = 256;

// partial[j * nchunks + c] = sum over rows [c * chunk, (c + 1) * chunk) of u_j . v_j
__global__ void __launch_bounds__(kDotThreads)
    k_coldot(int64_t n, int64_t chunk, int nchunks, const double* __restrict__ U, const double* __restrict__ V,
             int64_t ld, double* __restrict__ partial) {
    const int c = blockIdx.x, j = blockIdx.y;
    const int64_t r0 = (int64_t)c * chunk, r1 = min(n, r0 + chunk);
    const double* u = U + (int64_t)j * ld;
    const double* v = V + (int64_t)j * ld;
    double acc = 0.0;
    for (int64_t p = r0 + threadIdx.x; p < r1; p += kDotThreads) acc = fma(__ldg(u + p), __ldg(v + p), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[kDotThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kDotThreads / 32; ++w) s += red[w];
        partial[(int64_t)j * nchunks + c] = s;
    }
}

// out[j] = the chunk sums of column j added in a fixed order; act[j] &= (out[j] > 0).  One warp
// per column.
__global__ void k_dot_finalize(int b, int nchunks, const double* __restrict__ partial, double* __restrict__ out,
                               int* __restrict__ act) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= b) return;
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) s += partial[(int64_t)j * nchunks + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane) return;
    out[j] = s;
    if (!(s > 0.0)) act[j] = 0;
}

__global__ void k_fill_int(int b, int v, int* __restrict__ a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < b) a[j] = v;
}

// e_j += alpha_j p_j, r_j -= alpha_j (A p)_j with alpha_j = rz_j / pap_j on active columns.
__global__ void k_pcg_er(int64_t n, int b, const double* __restrict__ rz, const double* __restrict__ pap,
                         const int* __restrict__ act, double* __restrict__ E, double* __restrict__ R,
                         const double* __restrict__ P, const double* __restrict__ AP, int64_t ld) {
    const int j = blockIdx.y;
    if (!act[j]) return;
    const double alpha = rz[j] / pap[j];
    const int64_t off = (int64_t)j * ld;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        E[off + p] = fma(alpha, P[off + p], E[off + p]);
        R[off + p] = fma(-alpha, AP[off + p], R[off + p]);
    }
}

// p_j = z_j + beta_j p_j with beta_j = rz_new_j / rz_j on active columns.
__global__ void k_pcg_p(int64_t n, int b, const double* __restrict__ rz_new, const double* __restrict__ rz,
                        const int* __restrict__ act, double* __restrict__ P, const double* __restrict__ Z,
                        int64_t ld) {
    const int j = blockIdx.y;
    if (!act[j]) return;
    const double beta = rz_new[j] / rz[j];
    const int64_t off = (int64_t)j * ld;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        P[off + p] = fma(beta, P[off + p], Z[off + p]);
}

unsigned axpy_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256 * 8), 4 * kNumSMs)); }

}  // namespace

int pcg_chunks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8192), 2 * kNumSMs)); }

void launch_coldot(int64_t n, int b, const double* U, const double* V, int64_t ld, double* partial, double* out,
                   int* act, cudaStream_t st) {
    const int nchunks = pcg_chunks(n);
    const int64_t chunk = ceil_div(n, nchunks);
    k_coldot<<<dim3((unsigned)nchunks, (unsigned)b), kDotThreads, 0, st>>>(n, chunk, nchunks, U, V, ld, partial);
    LG_CHECK_LAUNCH();
    k_dot_finalize<<<(unsigned)ceil_div((int64_t)b * 32, 128), 128, 0, st>>>(b, nchunks, partial, out, act);
    LG_CHECK_LAUNCH();
}

void launch_fill_int(int b, int v, int* a, cudaStream_t st) {
    k_fill_int<<<(unsigned)ceil_div(b, 128), 128, 0, st>>>(b, v, a);
    LG_CHECK_LAUNCH();
}

void launch_pcg_er(int64_t n, int b, const double* rz, const double* pap, const int* act, double* E, double* R,
                   const double* P, const double* AP, int64_t ld, cudaStream_t st) {
    k_pcg_er<<<dim3(axpy_blocks(n), (unsigned)b), 256, 0, st>>>(n, b, rz, pap, act, E, R, P, AP, ld);
    LG_CHECK_LAUNCH();
}

void launch_pcg_p(int64_t n, int b, const double* rz_new, const double* rz, const int* act, double* P,
                  const double* Z, int64_t ld, cudaStream_t st) {
    k_pcg_p<<<dim3(axpy_blocks(n), (unsigned)b), 256, 0, st>>>(n, b, rz_new, rz, act, P, Z, ld);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
