// Variable-coefficient operator -div(kappa grad u) on the structured grid (unit spacing,
// Dirichlet: zero on the ghost layer), its V-cycle pieces and the eigenvalue gradient.
//
//   (A u)_p = scale * sum over the 6 faces f of p of kappa_f (u_p - u_q),   u_q = 0 outside.
//
// Face layout (float64, three consecutive parts, x fastest): x-faces (nx+1) * ny * nz, face
// (f, j, k) between cells (f-1, j, k) and (f, j, k); y-faces nx * (ny+1) * nz; z-faces
// nx * ny * (nz+1).  The diagonal D_p = sum of the 6 face values of p is formed on the fly.
//
// Coarse levels (the V-cycle's rediscretised operators) follow one reading: a coarse face takes
// the harmonic mean of the two fine faces it spans along its normal (one face where an
// even-sized axis is not nested at its far end), averages those line values over the fine lines
// at offsets -1, 0, +1 across it with weights 1/4, 1/2, 1/4 (lines outside the box dropped,
// weights renormalised), and is divided by 4 (mesh width 2h).  The coarsest level is solved
// exactly with a dense inverse built from its Cholesky factor.
//
// Eigenvalue gradient: for a unit eigenvector x_i of a simple eigenvalue,
// d lambda_i / d kappa_f = scale (x_i,p - x_i,q)^2 (first-order perturbation, dA/dkappa_f =
// scale (e_p - e_q)(e_p - e_q)^T); for weights w the kernel returns sum_i w_i of that.
#include <algorithm>

#include "common.cuh"

namespace lg {
namespace {

constexpr int kTX = 32, kTY = 4;

struct FaceIdx {
    int nx, ny, nz;
    int64_t oy, oz;    // offsets of the y- and z-face parts
    __host__ __device__ FaceIdx(const Grid3& g)
        : nx(g.nx), ny(g.ny), nz(g.nz), oy((int64_t)(g.nx + 1) * g.ny * g.nz),
          oz(oy + (int64_t)g.nx * (g.ny + 1) * g.nz) {}
    __host__ __device__ int64_t x(int f, int j, int k) const { return f + (int64_t)(nx + 1) * (j + (int64_t)ny * k); }
    __host__ __device__ int64_t y(int i, int f, int k) const { return oy + i + (int64_t)nx * (f + (int64_t)(ny + 1) * k); }
    __host__ __device__ int64_t z(int i, int j, int f) const { return oz + i + (int64_t)nx * (j + (int64_t)ny * f); }
};

// mode 0: y = scale (D x - N x)                        (SpMV, the products A X and A W)
// mode 1: y = (1 - w) x + w (z / (scale D) + N x / D)  (weighted Jacobi on e = x with r = z)
// mode 2: y = z - scale (D x - N x)                    (residual r - A e)
// mode 3: y = w z / (scale D)                          (first Jacobi sweep from e = 0)
template <int MODE>
__global__ void __launch_bounds__(kTX* kTY)
    k_vc_sweep(Grid3 g, int zchunk, int nzc, const double* __restrict__ kap, double scale, double w,
               const double* __restrict__ x, int64_t ldx, const double* __restrict__ z, int64_t ldz,
               double* __restrict__ y, int64_t ldy) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    if (i >= g.nx || j >= g.ny) return;
    const FaceIdx F(g);
    const int k0 = kc * zchunk, k1 = min(k0 + zchunk, g.nz);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const double* xc = x + (int64_t)col * ldx;
    const double* zc = z ? z + (int64_t)col * ldz : nullptr;
    double* yc = y + (int64_t)col * ldy;
    int64_t p = i + sy * (j + (int64_t)g.ny * k0);
    double xm = (MODE != 3 && k0 > 0) ? __ldg(xc + p - sz) : 0.0;
    double x0 = MODE != 3 ? __ldg(xc + p) : 0.0;
    double kzm = __ldg(kap + F.z(i, j, k0));
    for (int k = k0; k < k1; ++k, p += sz) {
        const double kzp = __ldg(kap + F.z(i, j, k + 1));
        const double kxl = __ldg(kap + F.x(i, j, k)), kxr = __ldg(kap + F.x(i + 1, j, k));
        const double kyd = __ldg(kap + F.y(i, j, k)), kyu = __ldg(kap + F.y(i, j + 1, k));
        const double d = ((kxl + kxr) + (kyd + kyu)) + (kzm + kzp);
        double v;
        if (MODE == 3) {
            v = w * __ldg(zc + p) / (scale * d);
        } else {
            const double xp = (k + 1 < g.nz) ? __ldg(xc + p + sz) : 0.0;
            double nb = kzm * xm + kzp * xp;
            if (i > 0) nb = fma(kxl, __ldg(xc + p - 1), nb);
            if (i + 1 < g.nx) nb = fma(kxr, __ldg(xc + p + 1), nb);
            if (j > 0) nb = fma(kyd, __ldg(xc + p - sy), nb);
            if (j + 1 < g.ny) nb = fma(kyu, __ldg(xc + p + sy), nb);
            if (MODE == 0) v = scale * fma(d, x0, -nb);
            else if (MODE == 2) v = __ldg(zc + p) - scale * fma(d, x0, -nb);
            else v = (1.0 - w) * x0 + w * (__ldg(zc + p) / scale + nb) / d;
            xm = x0;
            x0 = xp;
        }
        yc[p] = v;
        kzm = kzp;
    }
}

// Coarse face values (one thread per coarse face), reading of the file header.
__device__ double vc_line(const double* kap, const FaceIdx& Ff, int axis, int Fc, int a, int b, int nf_axis) {
    // harmonic mean along the normal of fine faces 2 Fc and 2 Fc + 1 at fine line (a, b)
    auto face = [&](int f) -> double {
        if (axis == 0) return __ldg(kap + Ff.x(f, a, b));
        if (axis == 1) return __ldg(kap + Ff.y(a, f, b));
        return __ldg(kap + Ff.z(a, b, f));
    };
    const int f0 = 2 * Fc, f1 = 2 * Fc + 1;
    if (f1 <= nf_axis) return 2.0 / (1.0 / face(f0) + 1.0 / face(f1));
    return face(f0);
}

__global__ void k_vc_coarsen(Grid3 gf, Grid3 gc, const double* __restrict__ kf, double* __restrict__ kc) {
    const FaceIdx Ff(gf), Fc(gc);
    const int64_t total = Fc.oz + (int64_t)gc.nx * gc.ny * (gc.nz + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int axis, F, A, B, na, nb, nfa, nfb, nf_axis;
        if (t < Fc.oy) {            // x-face (F, J, K): across axes y (J), z (K)
            axis = 0;
            F = (int)(t % (gc.nx + 1));
            A = (int)((t / (gc.nx + 1)) % gc.ny);
            B = (int)(t / ((int64_t)(gc.nx + 1) * gc.ny));
            nfa = gf.ny; nfb = gf.nz; nf_axis = gf.nx;
        } else if (t < Fc.oz) {     // y-face (I, F, K): across x (I), z (K)
            const int64_t u = t - Fc.oy;
            axis = 1;
            A = (int)(u % gc.nx);
            F = (int)((u / gc.nx) % (gc.ny + 1));
            B = (int)(u / ((int64_t)gc.nx * (gc.ny + 1)));
            nfa = gf.nx; nfb = gf.nz; nf_axis = gf.ny;
        } else {                    // z-face (I, J, F): across x (I), y (J)
            const int64_t u = t - Fc.oz;
            axis = 2;
            A = (int)(u % gc.nx);
            B = (int)((u / gc.nx) % gc.ny);
            F = (int)(u / ((int64_t)gc.nx * gc.ny));
            nfa = gf.nx; nfb = gf.ny; nf_axis = gf.nz;
        }
        (void)na; (void)nb;
        const double wt[3] = {0.25, 0.5, 0.25};
        double acc = 0.0, tot = 0.0;
        for (int db = -1; db <= 1; ++db) {
            const int b = 2 * B + 1 + db;
            if (b < 0 || b >= nfb) continue;
            for (int da = -1; da <= 1; ++da) {
                const int a = 2 * A + 1 + da;
                if (a < 0 || a >= nfa) continue;
                const double wgt = wt[da + 1] * wt[db + 1];
                acc += wgt * vc_line(kf, Ff, axis, F, a, b, nf_axis);
                tot += wgt;
            }
        }
        kc[t] = acc / tot / 4.0;
    }
}

// Dense matrix of the operator on a (small) grid, column-major n x n.
__global__ void k_vc_dense(Grid3 g, const double* __restrict__ kap, double scale, double* __restrict__ A) {
    const int64_t n = g.n();
    const FaceIdx F(g);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x)
        A[t] = 0.0;
    __syncthreads();
    // one thread per row p (the grid is small: one block suffices and keeps the order simple)
    for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
        const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
        const double kxl = kap[F.x(i, j, k)], kxr = kap[F.x(i + 1, j, k)];
        const double kyd = kap[F.y(i, j, k)], kyu = kap[F.y(i, j + 1, k)];
        const double kzd = kap[F.z(i, j, k)], kzu = kap[F.z(i, j, k + 1)];
        A[p + n * p] = scale * (((kxl + kxr) + (kyd + kyu)) + (kzd + kzu));
        if (i > 0) A[p + n * (p - 1)] = -scale * kxl;
        if (i + 1 < g.nx) A[p + n * (p + 1)] = -scale * kxr;
        if (j > 0) A[p + n * (p - g.nx)] = -scale * kyd;
        if (j + 1 < g.ny) A[p + n * (p + g.nx)] = -scale * kyu;
        if (k > 0) A[p + n * (p - (int64_t)g.nx * g.ny)] = -scale * kzd;
        if (k + 1 < g.nz) A[p + n * (p + (int64_t)g.nx * g.ny)] = -scale * kzu;
    }
}

// In-place lower Cholesky of the column-major n x n matrix A (one block); sets *fail on a
// non-positive pivot.
__global__ void __launch_bounds__(1024) k_dense_chol(int n, double* A, int* fail) {
    __shared__ double rinv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double piv = A[k + (int64_t)n * k];
            if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
            else { const double l = sqrt(piv); A[k + (int64_t)n * k] = l; rinv = 1.0 / l; }
        }
        __syncthreads();
        if (bad) { if (threadIdx.x == 0) *fail = 1; return; }
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (int64_t)n * k] *= rinv;
        __syncthreads();
        const int rem = n - k - 1;
        for (int64_t e = threadIdx.x; e < (int64_t)rem * rem; e += blockDim.x) {
            const int i = k + 1 + (int)(e % rem), jj = k + 1 + (int)(e / rem);
            if (i >= jj) A[i + (int64_t)n * jj] -= A[i + (int64_t)n * k] * A[jj + (int64_t)n * k];
        }
        __syncthreads();
    }
}

// Column j of A^-1 from the lower Cholesky factor L (block j; one thread does the two
// triangular solves, the block's other threads copy the result).
__global__ void k_dense_inv_col(int n, const double* __restrict__ L, double* __restrict__ work,
                                double* __restrict__ Ainv) {
    const int jc = blockIdx.x;
    double* y = work + (int64_t)jc * n;
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {          // L y = e_j
            double s = (i == jc) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i + (int64_t)n * k] * y[k];
            y[i] = s / L[i + (int64_t)n * i];
        }
        for (int i = n - 1; i >= 0; --i) {     // L^T x = y
            double s = y[i];
            for (int k = i + 1; k < n; ++k) s -= L[k + (int64_t)n * i] * y[k];
            y[i] = s / L[i + (int64_t)n * i];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) Ainv[i + (int64_t)n * jc] = y[i];
}

// e[:, c] = Ainv r[:, c] (block per column).
__global__ void k_dense_apply(int n, const double* __restrict__ Ainv, const double* __restrict__ r, int64_t ldr,
                              double* __restrict__ e, int64_t lde) {
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(Ainv[i + (int64_t)n * k], __ldg(r + (int64_t)c * ldr + k), s);
        e[(int64_t)c * lde + i] = s;
    }
}

struct Weights {
    double w[kMaxM];
};

// grad[f] = scale * sum_i w_i (x_i,q - x_i,p)^2 over the m columns of X (zero outside the box).
__global__ void k_vc_grad(Grid3 g, int m, Weights wt, double scale, const double* __restrict__ X, int64_t ldx,
                          double* __restrict__ grad) {
    const FaceIdx F(g);
    const int64_t total = F.oz + (int64_t)g.nx * g.ny * (g.nz + 1);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t pa = -1, pb = -1;     // cells on the two sides (-1: ghost)
        if (t < F.oy) {
            const int f = (int)(t % (g.nx + 1));
            const int j = (int)((t / (g.nx + 1)) % g.ny), k = (int)(t / ((int64_t)(g.nx + 1) * g.ny));
            const int64_t base = sy * j + sz * k;
            if (f > 0) pa = base + f - 1;
            if (f < g.nx) pb = base + f;
        } else if (t < F.oz) {
            const int64_t u = t - F.oy;
            const int i = (int)(u % g.nx), f = (int)((u / g.nx) % (g.ny + 1)), k = (int)(u / ((int64_t)g.nx * (g.ny + 1)));
            const int64_t base = i + sz * k;
            if (f > 0) pa = base + sy * (f - 1);
            if (f < g.ny) pb = base + sy * f;
        } else {
            const int64_t u = t - F.oz;
            const int i = (int)(u % g.nx), j = (int)((u / g.nx) % g.ny), f = (int)(u / ((int64_t)g.nx * g.ny));
            const int64_t base = i + sy * j;
            if (f > 0) pa = base + sz * (f - 1);
            if (f < g.nz) pb = base + sz * f;
        }
        double s = 0.0;
        for (int c = 0; c < m; ++c) {
            const double* xc = X + (int64_t)c * ldx;
            const double d = (pb >= 0 ? __ldg(xc + pb) : 0.0) - (pa >= 0 ? __ldg(xc + pa) : 0.0);
            s = fma(wt.w[c], d * d, s);
        }
        grad[t] = scale * s;
    }
}

__host__ __device__ inline int vc_zchunk(int nz) { return nz >= 128 ? 16 : (nz >= 32 ? 4 : (nz >= 8 ? 2 : nz)); }

}  // namespace

int64_t vc_num_faces(const Grid3& g) {
    return (int64_t)(g.nx + 1) * g.ny * g.nz + (int64_t)g.nx * (g.ny + 1) * g.nz + (int64_t)g.nx * g.ny * (g.nz + 1);
}

void launch_vc_sweep(const Grid3& g, int mode, int ncols, const double* kap, double scale, double w,
                     const double* x, int64_t ldx, const double* z, int64_t ldz, double* y, int64_t ldy,
                     cudaStream_t st) {
    if (ncols <= 0) return;
    const int zc = vc_zchunk(g.nz);
    const int nzc = (int)ceil_div(g.nz, zc);
    dim3 grid((unsigned)ceil_div(g.nx, kTX), (unsigned)ceil_div(g.ny, kTY), (unsigned)(nzc * ncols));
    dim3 block(kTX, kTY);
    switch (mode) {
        case 0: k_vc_sweep<0><<<grid, block, 0, st>>>(g, zc, nzc, kap, scale, w, x, ldx, z, ldz, y, ldy); break;
        case 1: k_vc_sweep<1><<<grid, block, 0, st>>>(g, zc, nzc, kap, scale, w, x, ldx, z, ldz, y, ldy); break;
        case 2: k_vc_sweep<2><<<grid, block, 0, st>>>(g, zc, nzc, kap, scale, w, x, ldx, z, ldz, y, ldy); break;
        default: k_vc_sweep<3><<<grid, block, 0, st>>>(g, zc, nzc, kap, scale, w, x, ldx, z, ldz, y, ldy); break;
    }
    LG_CHECK_LAUNCH();
}

void launch_vc_coarsen(const Grid3& gf, const Grid3& gc, const double* kf, double* kc, cudaStream_t st) {
    const int64_t total = vc_num_faces(gc);
    k_vc_coarsen<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, st>>>(gf, gc, kf, kc);
    LG_CHECK_LAUNCH();
}

void launch_vc_coarse_inverse(const Grid3& g, const double* kap, double scale, double* A, double* work,
                              double* Ainv, int* fail, cudaStream_t st) {
    const int n = (int)g.n();
    k_vc_dense<<<1, 1024, 0, st>>>(g, kap, scale, A);
    LG_CHECK_LAUNCH();
    k_dense_chol<<<1, 1024, 0, st>>>(n, A, fail);
    LG_CHECK_LAUNCH();
    k_dense_inv_col<<<n, 128, 0, st>>>(n, A, work, Ainv);
    LG_CHECK_LAUNCH();
}

void launch_dense_apply(int n, int ncols, const double* Ainv, const double* r, int64_t ldr, double* e, int64_t lde,
                        cudaStream_t st) {
    if (ncols <= 0) return;
    k_dense_apply<<<ncols, 128, 0, st>>>(n, Ainv, r, ldr, e, lde);
    LG_CHECK_LAUNCH();
}

void launch_vc_grad(const Grid3& g, int m, const double* w, double scale, const double* X, int64_t ldx,
                    double* grad, cudaStream_t st) {
    Weights wt{};
    for (int i = 0; i < m && i < kMaxM; ++i) wt.w[i] = w[i];
    const int64_t total = vc_num_faces(g);
    k_vc_grad<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), (int64_t)kNumSMs * 16), 256, 0, st>>>(
        g, m, wt, scale, X, ldx, grad);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
