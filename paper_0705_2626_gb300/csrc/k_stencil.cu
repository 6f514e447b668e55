// Stencil-family kernels: the block 7-point SpMV (Section 2.2) and the
// kernels of the multigrid V-cycle that serves as the preconditioner T (the preconditioning).
//
// All of them are one generic structured sweep
//     y = a*x + b*(sum of the six neighbours of x) [+ c*z]          (zero outside the grid)
// which covers
//     SpMV            y = A x            a = 6s,              b = -s
//     Jacobi sweep    e' = e + w D^-1 (r - A e)
//                        = (1-w) e + (w/6) nb(e) + (w/(6s)) r        (D = 6s)
//     first sweep     from e = 0 the first two sweeps fold into one:
//                     e2 = alpha(2-w) r + (alpha w/6) nb(r),   alpha = w/(6s)
//     residual        res = r - A e = -6s e + s nb(e) + r
// Layout: column-major blocks, point p = i + nx*(j + ny*k).  Each thread owns one (i, j)
// line and marches along k over a chunk of planes, carrying the k-1, k, k+1 values in
// registers; in-plane neighbours come through L1.  Storage is float64, float32 or bfloat16;
// arithmetic is float64 for float64 data (bound by GB300's FP64 pipe, 7-8 instructions per
// point) and float32 otherwise (bound by HBM).
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "dtype.cuh"

namespace lg {
namespace {

constexpr int kTX = 32, kTY = 4;

// Planes per thread along k: long runs on large grids (register reuse of the k-1 / k / k+1
// values), short runs on the small coarse grids, which live in L2 and need the parallelism.
__host__ __device__ inline int zchunk_for(int nz) { return nz >= 128 ? 16 : (nz >= 32 ? 4 : (nz >= 8 ? 2 : nz)); }

template <typename T, bool HAS_Z>
__global__ void __launch_bounds__(kTX* kTY)
    k_stencil_axpby(Grid3 g, int zchunk, int nzc, typename Acc<T>::type a, typename Acc<T>::type b,
                    const T* __restrict__ x, int64_t ldx, typename Acc<T>::type c,
                    const T* __restrict__ z, int64_t ldz, T* __restrict__ y, int64_t ldy) {
    using C = typename Acc<T>::type;
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    if (i >= g.nx || j >= g.ny) return;
    const int k0 = kc * zchunk;
    const int k1 = min(k0 + zchunk, g.nz);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const T* xc = x + (int64_t)col * ldx;
    const T* zc = HAS_Z ? z + (int64_t)col * ldz : nullptr;
    T* yc = y + (int64_t)col * ldy;
    int64_t p = i + sy * (j + (int64_t)g.ny * k0);
    C xm = (k0 > 0) ? ld_as(xc + p - sz) : C(0);
    C x0 = ld_as(xc + p);
    const bool hasl = i > 0, hasr = i + 1 < g.nx, hasd = j > 0, hasu = j + 1 < g.ny;
    for (int k = k0; k < k1; ++k, p += sz) {
        const C xp = (k + 1 < g.nz) ? ld_as(xc + p + sz) : C(0);
        C v;
        if constexpr (sizeof(C) == 8) {
            C nb = xm + xp;
            if (hasl) nb += ld_as(xc + p - 1);
            if (hasr) nb += ld_as(xc + p + 1);
            if (hasd) nb += ld_as(xc + p - sy);
            if (hasu) nb += ld_as(xc + p + sy);
            v = fma(b, nb, a * x0);
        } else {
            // float32 arithmetic: y = (a + 6b) x - b * sum_q (x - x_q).  For a smooth field the
            // neighbour differences are exact (Sterbenz), so A x = s sum (x - x_q) keeps its
            // relative accuracy instead of losing it to the cancellation in 6x - sum x_q.
            C d = (x0 - xm) + (x0 - xp);
            d += hasl ? x0 - ld_as(xc + p - 1) : x0;
            d += hasr ? x0 - ld_as(xc + p + 1) : x0;
            d += hasd ? x0 - ld_as(xc + p - sy) : x0;
            d += hasu ? x0 - ld_as(xc + p + sy) : x0;
            v = fma(-b, d, (a + C(6) * b) * x0);
        }
        if (HAS_Z) v = fma(c, ld_as(zc + p), v);
        st_as(yc + p, v);
        xm = x0;
        x0 = xp;
    }
}

// Float32 or bfloat16 storage with nx divisible by 4: each thread owns 4 consecutive points of an
// x-row (one 16- or 8-byte vector) over a run of planes along k, so a point costs about 1.25 load
// instructions instead of 6.  Float32 arithmetic, the difference form of the branch above with
// the neighbours added in the same order.
__device__ __forceinline__ float4 ld4v(const float* q) { return __ldg(reinterpret_cast<const float4*>(q)); }
__device__ __forceinline__ float4 ld4v(const __nv_bfloat16* q) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(q));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ void st4v(float* q, const float (&o)[4]) {
    *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4v(__nv_bfloat16* q, const float (&o)[4]) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]), hi = __floats2bfloat162_rn(o[2], o[3]);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned*>(&lo);
    u.y = *reinterpret_cast<const unsigned*>(&hi);
    *reinterpret_cast<uint2*>(q) = u;
}

// A thread's run of ZC planes issues all of its loads -- the ZC + 2 planes of its x vector, the
// y-neighbour vectors, the x-neighbour scalars and the z vectors -- before any arithmetic, so the
// run waits for one memory round trip instead of one per plane.
template <typename T, bool HAS_Z, int ZC>
__global__ void __launch_bounds__(kTX* kTY)
    k_stencil_v4(Grid3 g, int nzc, float a, float b, const T* __restrict__ x, int64_t ldx, float c,
                 const T* __restrict__ z, int64_t ldz, T* __restrict__ y, int64_t ldy) {
    const int nx4 = g.nx >> 2;
    const int i4 = blockIdx.x * blockDim.x + threadIdx.x;   // block (32, 4), or (16, 8) / (8, 16) for short rows
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    if (i4 >= nx4 || j >= g.ny) return;
    const int i0 = 4 * i4;
    const int k0 = kc * ZC;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const T* xc = x + (int64_t)col * ldx;
    const T* zc = HAS_Z ? z + (int64_t)col * ldz : nullptr;
    T* yc = y + (int64_t)col * ldy;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t p0 = i0 + sy * (j + (int64_t)g.ny * k0);
    const bool hasl = i0 > 0, hasr = i0 + 4 < g.nx, hasd = j > 0, hasu = j + 1 < g.ny;
    float4 xs[ZC + 2], yd[ZC], yu[ZC], zz[ZC];     // xs[q]: plane k0 - 1 + q
    float ls[ZC], rs[ZC];
#pragma unroll
    for (int q = 0; q < ZC + 2; ++q) {
        const int k = k0 - 1 + q;
        xs[q] = (k >= 0 && k < g.nz) ? ld4v(xc + p0 + (int64_t)(q - 1) * sz) : zero;
    }
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
        const bool in = k0 + q < g.nz;
        const int64_t p = p0 + (int64_t)q * sz;
        yd[q] = in && hasd ? ld4v(xc + p - sy) : zero;
        yu[q] = in && hasu ? ld4v(xc + p + sy) : zero;
        ls[q] = in && hasl ? (float)ld_as(xc + p - 1) : 0.f;
        rs[q] = in && hasr ? (float)ld_as(xc + p + 4) : 0.f;
        zz[q] = in && HAS_Z ? ld4v(zc + p) : zero;
    }
    const float a6 = a + 6.f * b;
#pragma unroll
    for (int q = 0; q < ZC; ++q) {
        if (k0 + q >= g.nz) break;
        const float4 xm = xs[q], x0 = xs[q + 1], xp = xs[q + 2];
        const float cx[6] = {ls[q], x0.x, x0.y, x0.z, x0.w, rs[q]};
        const float m_[4] = {xm.x, xm.y, xm.z, xm.w}, p_[4] = {xp.x, xp.y, xp.z, xp.w};
        const float d_[4] = {yd[q].x, yd[q].y, yd[q].z, yd[q].w}, u_[4] = {yu[q].x, yu[q].y, yu[q].z, yu[q].w};
        const float z_[4] = {zz[q].x, zz[q].y, zz[q].z, zz[q].w};
        float o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float xv = cx[e + 1];
            float d = (xv - m_[e]) + (xv - p_[e]);
            d += xv - cx[e];
            d += xv - cx[e + 2];
            d += xv - d_[e];
            d += xv - u_[e];
            float v = fmaf(-b, d, a6 * xv);
            if (HAS_Z) v = fmaf(c, z_[e], v);
            o[e] = v;
        }
        st4v(yc + p0 + (int64_t)q * sz, o);
    }
}

// Full weighting: coarse point (I, J, K) (0-based) sits on fine (2I+1, 2J+1, 2K+1);
// weights 1, 1/2 per axis for offsets 0, +-1, overall factor 1/8 (R = P^T / 8).
template <typename TF, typename TC>
__global__ void __launch_bounds__(kTX* kTY)
    k_restrict(Grid3 gf, Grid3 gc, const TF* __restrict__ rf, int64_t ldf, TC* __restrict__ rc,
               int64_t ldc) {
    using C = typename Acc<TF>::type;
    const int I = blockIdx.x * kTX + threadIdx.x;
    const int J = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / gc.nz;
    const int K = blockIdx.z - col * gc.nz;
    if (I >= gc.nx || J >= gc.ny) return;
    const TF* f = rf + (int64_t)col * ldf;
    const int fi = 2 * I + 1, fj = 2 * J + 1, fk = 2 * K + 1;
    C s = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = fk + dz;
        if (kk >= gf.nz) continue;
        const C wz = dz == 0 ? C(1) : C(0.5);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int jj = fj + dy;
            if (jj >= gf.ny) continue;
            const C wzy = wz * (dy == 0 ? C(1) : C(0.5));
            const int64_t row = (int64_t)gf.nx * (jj + (int64_t)gf.ny * kk);
            C t = ld_as(f + row + fi);
            if (fi - 1 >= 0) t = fma(C(0.5), ld_as(f + row + fi - 1), t);
            if (fi + 1 < gf.nx) t = fma(C(0.5), ld_as(f + row + fi + 1), t);
            s = fma(wzy, t, s);
        }
    }
    st_as(rc + (int64_t)col * ldc + I + (int64_t)gc.nx * (J + (int64_t)gc.ny * K), C(0.125) * s);
}

// The same full weighting for float32 / bfloat16 fine levels with nx divisible by 4: a thread owns
// the coarse points (2 I2, J) and (2 I2 + 1, J) -- fine x 4 I2 .. 4 I2 + 4, one vector and one
// scalar per fine row -- and marches along K, reusing the weighted sum of the fine plane 2K + 2 as
// that of plane 2(K + 1): about 6 loads per coarse point instead of 27.
template <typename TF, typename TC>
__global__ void __launch_bounds__(kTX* kTY)
    k_restrict_v4(Grid3 gf, Grid3 gc, int kchunk, int nkc, const TF* __restrict__ rf, int64_t ldf,
                  TC* __restrict__ rc, int64_t ldc) {
    const int I2 = blockIdx.x * blockDim.x + threadIdx.x;   // block shape as for the stencil rows
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int col = blockIdx.z / nkc;
    const int kc = blockIdx.z - col * nkc;
    const int I0 = 2 * I2;
    if (I0 >= gc.nx || J >= gc.ny) return;
    const int K0 = kc * kchunk, K1 = min(K0 + kchunk, gc.nz);
    const int64_t sy = gf.nx, sz = (int64_t)gf.nx * gf.ny;
    const TF* f = rf + (int64_t)col * ldf;
    const int fx = 4 * I2;                         // fine x of the vector: 4 I2 .. 4 I2 + 3
    const bool has4 = fx + 4 < gf.nx;              // fine x 4 I2 + 4 (right neighbour of the second point)
    const int fy = 2 * J;                          // fine rows 2J .. 2J + 2
    const bool hasy2 = fy + 2 < gf.ny;
    // x- and y-weighted sums of fine plane z for the two coarse points
    auto plane = [&](int z, float& c0, float& c1) {
        c0 = c1 = 0.f;
        if (z >= gf.nz) return;
        const TF* pl = f + (int64_t)z * sz + fx;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            if (dy == 2 && !hasy2) break;
            const TF* row = pl + (int64_t)(fy + dy) * sy;
            const float4 v = ld4v(row);
            const float e = has4 ? (float)ld_as(row + 4) : 0.f;
            const float a0 = fmaf(0.5f, v.x + v.z, v.y);          // fine 4I2+1 with 4I2, 4I2+2
            const float a1 = fmaf(0.5f, v.z + e, v.w);            // fine 4I2+3 with 4I2+2, 4I2+4
            const float wy = dy == 1 ? 1.f : 0.5f;
            c0 = fmaf(wy, a0, c0);
            c1 = fmaf(wy, a1, c1);
        }
    };
    const bool two = I0 + 1 < gc.nx;
    TC* out = rc + (int64_t)col * ldc + I0 + (int64_t)gc.nx * J;
    float lo0, lo1;
    plane(2 * K0, lo0, lo1);
    for (int K = K0; K < K1; ++K) {
        float m0, m1, h0, h1;
        plane(2 * K + 1, m0, m1);
        plane(2 * K + 2, h0, h1);
        const int64_t o = (int64_t)gc.nx * gc.ny * K;
        st_as(out + o, 0.125f * (0.5f * (lo0 + h0) + m0));
        if (two) st_as(out + o + 1, 0.125f * (0.5f * (lo1 + h1) + m1));
        lo0 = h0;
        lo1 = h1;
    }
}

// Prolongation by coarse cells: cell (Cx, Cy, Cz), 0 <= C <= nc per axis, lies between the
// coarse points C and C+1 (1-based; 0 and nc+1 are the zero boundary) and owns the fine points
// 2C+1 (midpoint, weight 1/2 each) and 2C+2 (on coarse C+1, weight 1) of each axis that exist.
// A thread owns a (Cx, Cy) column of cells and marches along Cz carrying the lower coarse plane,
// so each coarse value is loaded about once per 8 fine points it feeds.
template <typename TC, typename TF>
__global__ void __launch_bounds__(kTX* kTY)
    k_prolong_add(Grid3 gf, Grid3 gc, int zchunk, int nzc, const TC* __restrict__ ec, int64_t ldc,
                  TF* __restrict__ ef, int64_t ldf) {
    using C = typename Acc<TF>::type;
    const int cx = blockIdx.x * kTX + threadIdx.x;
    const int cy = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    if (cx > gc.nx || cy > gc.ny) return;
    const int z0 = kc * zchunk;
    const int z1 = min(z0 + zchunk, gc.nz + 1);
    const TC* c = ec + (int64_t)col * ldc;
    TF* f = ef + (int64_t)col * ldf;
    const int64_t csy = gc.nx, csz = (int64_t)gc.nx * gc.ny;
    const int64_t fsy = gf.nx, fsz = (int64_t)gf.nx * gf.ny;
    // coarse value at 1-based (X, Y, Z), zero outside 1..nc
    auto cv = [&](int X, int Y, int Z) -> C {
        if (X < 1 || X > gc.nx || Y < 1 || Y > gc.ny || Z < 1 || Z > gc.nz) return C(0);
        return C(ld_as(c + (X - 1) + csy * (Y - 1) + csz * (Z - 1)));
    };
    // lo[b][a]: plane Z = Cz, hi[b][a]: plane Z = Cz + 1; a, b select X = cx + a, Y = cy + b
    C lo[2][2], hi[2][2];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) lo[b][a] = cv(cx + a, cy + b, z0);
    for (int cz = z0; cz < z1; ++cz) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) hi[b][a] = cv(cx + a, cy + b, cz + 1);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const int fz = 2 * cz + dz;           // 0-based fine index
            if (fz >= gf.nz) break;
            C pz[2][2];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) pz[b][a] = dz ? hi[b][a] : C(0.5) * (lo[b][a] + hi[b][a]);
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int fy = 2 * cy + dy;
                if (fy >= gf.ny) break;
                const C py0 = dy ? pz[1][0] : C(0.5) * (pz[0][0] + pz[1][0]);
                const C py1 = dy ? pz[1][1] : C(0.5) * (pz[0][1] + pz[1][1]);
                const int64_t row = fsy * fy + fsz * fz;
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const int fx = 2 * cx + dx;
                    if (fx >= gf.nx) break;
                    const C v = dx ? py1 : C(0.5) * (py0 + py1);
                    TF* q = f + row + fx;
                    st_as(q, C(ld_as(q)) + v);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) lo[b][a] = hi[b][a];
    }
}

// The same prolongation for float32 / bfloat16 fine levels with nx divisible by 4: a thread owns
// the fine x-points 4t .. 4t+3 of the fine rows 2cy, 2cy+1 and marches along the cells' z.  Fine
// x 4t, 4t+1, 4t+2, 4t+3 interpolate the coarse x-points 2t, 2t+1, 2t+2 (1-based; one 2-vector
// and one scalar per coarse row); each coarse row is interpolated in x once and the two rows and
// two planes of a cell are then combined in y and z, so a fine vector costs one load and one
// store.
__device__ __forceinline__ float2 ld2v(const float* q) { return __ldg(reinterpret_cast<const float2*>(q)); }
__device__ __forceinline__ float2 ld2v(const __nv_bfloat16* q) {
    const unsigned u = __ldg(reinterpret_cast<const unsigned*>(q));
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

template <typename TC, typename TF>
__global__ void __launch_bounds__(kTX* kTY)
    k_prolong_v4(Grid3 gf, Grid3 gc, int zchunk, int nzc, const TC* __restrict__ ec, int64_t ldc,
                 TF* __restrict__ ef, int64_t ldf) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    if (4 * t >= gf.nx || 2 * cy >= gf.ny) return;
    const int ncz = (gf.nz + 1) / 2;               // cells along z that own fine planes
    const int z0 = kc * zchunk, z1 = min(z0 + zchunk, ncz);
    const TC* c = ec + (int64_t)col * ldc;
    TF* f = ef + (int64_t)col * ldf;
    const int64_t csz = (int64_t)gc.nx * gc.ny;
    const int64_t fsy = gf.nx, fsz = (int64_t)gf.nx * gf.ny;
    // coarse row (Y, Z) (1-based, zero outside 1..nc) interpolated to the fine x 4t .. 4t+3
    auto xrow = [&](int Y, int Z, float (&v)[4]) {
        if (Y < 1 || Y > gc.ny || Z < 1 || Z > gc.nz) {
            v[0] = v[1] = v[2] = v[3] = 0.f;
            return;
        }
        const TC* row = c + (int64_t)gc.nx * (Y - 1) + csz * (Z - 1);
        const float2 ab = ld2v(row + 2 * t);       // X = 2t+1, 2t+2
        const float m = t > 0 ? (float)ld_as(row + 2 * t - 1) : 0.f;   // X = 2t
        v[0] = 0.5f * (m + ab.x);
        v[1] = ab.x;
        v[2] = 0.5f * (ab.x + ab.y);
        v[3] = ab.y;
    };
    float lo[2][4], hi[2][4];                     // [Y = cy, cy+1][x] on planes Z = cz (lo), cz+1 (hi)
    xrow(cy, z0, lo[0]);
    xrow(cy + 1, z0, lo[1]);
    for (int cz = z0; cz < z1; ++cz) {
        xrow(cy, cz + 1, hi[0]);
        xrow(cy + 1, cz + 1, hi[1]);
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
            const int fz = 2 * cz + dz;
            if (fz >= gf.nz) break;
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const int fy = 2 * cy + dy;
                if (fy >= gf.ny) break;
                TF* q = f + fsz * fz + fsy * fy + 4 * t;
                const float4 old = ld4v(q);
                const float o4[4] = {old.x, old.y, old.z, old.w};
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float p0 = dz ? hi[0][e] : 0.5f * (lo[0][e] + hi[0][e]);
                    const float p1 = dz ? hi[1][e] : 0.5f * (lo[1][e] + hi[1][e]);
                    o[e] = o4[e] + (dy ? p1 : 0.5f * (p0 + p1));
                }
                st4v(q, o);
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int e = 0; e < 4; ++e) lo[r][e] = hi[r][e];
    }
}

// Coarsest-level exact solve.  The 7-point Dirichlet operator s*(6u - nb) on an
// nx x ny x nz box has the orthonormal eigenvectors Qz (x) Qy (x) Qx with
// Q_d[a][i] = sqrt(2/(n_d+1)) sin(pi (a+1)(i+1)/(n_d+1)) (symmetric, Q_d^2 = I) and the
// eigenvalues 4s (sin^2(pi(a+1)/(2(nx+1))) + ...), so A^-1 = Q diag(1/lambda) Q.
__global__ void k_coarse_setup(Grid3 g, double scale, double* tab) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    double* Qx = tab;
    double* Qy = Qx + nx * nx;
    double* Qz = Qy + ny * ny;
    double* lam = Qz + nz * nz;
    const int64_t total = (int64_t)nx * nx + ny * ny + nz * nz + g.n();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < (int64_t)nx * nx) {
            const int a = t / nx, i = t % nx;
            Qx[t] = sqrt(2.0 / (nx + 1)) * sinpi((double)((a + 1) * (i + 1)) / (nx + 1));
        } else if (t < (int64_t)nx * nx + ny * ny) {
            const int u = t - nx * nx, a = u / ny, i = u % ny;
            Qy[u] = sqrt(2.0 / (ny + 1)) * sinpi((double)((a + 1) * (i + 1)) / (ny + 1));
        } else if (t < (int64_t)nx * nx + ny * ny + nz * nz) {
            const int u = t - nx * nx - ny * ny, a = u / nz, i = u % nz;
            Qz[u] = sqrt(2.0 / (nz + 1)) * sinpi((double)((a + 1) * (i + 1)) / (nz + 1));
        } else {
            const int64_t p = t - (int64_t)nx * nx - ny * ny - nz * nz;
            const int a = p % nx, b = (p / nx) % ny, c = p / ((int64_t)nx * ny);
            const double sx = sinpi((double)(a + 1) / (2.0 * (nx + 1)));
            const double sy = sinpi((double)(b + 1) / (2.0 * (ny + 1)));
            const double sz = sinpi((double)(c + 1) / (2.0 * (nz + 1)));
            lam[p] = 4.0 * scale * (sx * sx + sy * sy + sz * sz);
        }
    }
}

// One 1-D transform pass along axis `ax` (0 = x, 1 = y, 2 = z): out = Q_ax applied to in.
__device__ void sine_pass(const Grid3& g, int ax, const double* __restrict__ Q,
                          const double* in, double* out) {
    const int n = g.nx * g.ny * g.nz;
    const int na = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
    const int stride = ax == 0 ? 1 : (ax == 1 ? g.nx : g.nx * g.ny);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int a = (p / stride) % na;           // output index along the axis
        const int base = p - a * stride;
        double s = 0.0;
        for (int i = 0; i < na; ++i) s = fma(__ldg(Q + a * na + i), in[base + i * stride], s);
        out[p] = s;
    }
    __syncthreads();
}

// The same pass with Q in shared memory (plain loads; the same order of operations).
__device__ void sine_pass_sm(const Grid3& g, int ax, const double* Q, const double* in, double* out) {
    const int n = g.nx * g.ny * g.nz;
    const int na = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
    const int stride = ax == 0 ? 1 : (ax == 1 ? g.nx : g.nx * g.ny);
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int a = (p / stride) % na;
        const int base = p - a * stride;
        double s = 0.0;
        for (int i = 0; i < na; ++i) s = fma(Q[a * na + i], in[base + i * stride], s);
        out[p] = s;
    }
    __syncthreads();
}

template <typename T>
__global__ void k_coarse_solve(Grid3 g, const double* __restrict__ tab, const T* __restrict__ r,
                               int64_t ldr, T* __restrict__ e, int64_t lde) {
    extern __shared__ double sm[];
    const int n = g.nx * g.ny * g.nz;
    double* u = sm;
    double* v = sm + n;
    const double* Qx = tab;
    const double* Qy = Qx + g.nx * g.nx;
    const double* Qz = Qy + g.ny * g.ny;
    const double* lam = Qz + g.nz * g.nz;
    const int col = blockIdx.x;
    for (int p = threadIdx.x; p < n; p += blockDim.x) u[p] = (double)ld_as(r + (int64_t)col * ldr + p);
    __syncthreads();
    sine_pass(g, 0, Qx, u, v);
    sine_pass(g, 1, Qy, v, u);
    sine_pass(g, 2, Qz, u, v);
    for (int p = threadIdx.x; p < n; p += blockDim.x) v[p] /= lam[p];
    __syncthreads();
    sine_pass(g, 0, Qx, v, u);
    sine_pass(g, 1, Qy, u, v);
    sine_pass(g, 2, Qz, v, u);
    for (int p = threadIdx.x; p < n; p += blockDim.x) st_as(e + (int64_t)col * lde + p, u[p]);
}

// ---------------------------------------------------------------- small levels, fused
// The coarse end of the V-cycle (every level with at most kFuseMaxPoints points and the levels
// below it) in one kernel: one thread block per column keeps all of its level vectors in shared
// memory (compute type C: float for float32 / bfloat16 storage, double for float64) and runs the
// same steps as the multi-kernel path -- fused first two pre-sweeps, Jacobi sweeps, residual,
// full-weighting restriction, exact sine-transform solve on the coarsest level, trilinear
// prolongation, post-sweeps -- separated by block barriers instead of kernel launches.
constexpr int kSmallThreads = 512;    // block of the fused small-level V-cycle (1024 measured slower)

struct SmallLevels {
    int nl;
    Grid3 g[kFuseMaxLevels];
    double s[kFuseMaxLevels];
    int off[kFuseMaxLevels];    // element offset of level l's three vectors (r, e, t)
};

// Threads of the block over the (i, j) lines of a level: when the block has more threads than a
// plane has lines, each line is split into nsplit runs along k.  A thread marches its run,
// carrying the k-1 / k / k+1 values in registers (one division per line instead of three per
// point).
struct SmLines {
    int P, nsplit, kper;
    __device__ SmLines(const Grid3& g) {
        P = g.nx * g.ny;
        nsplit = P >= (int)blockDim.x ? 1 : min(g.nz, (int)blockDim.x / P);
        kper = (g.nz + nsplit - 1) / nsplit;
    }
};

template <typename C>
__device__ void sm_axpby(const Grid3& g, C a, C b, const C* __restrict__ x, C c, const C* __restrict__ z,
                         C* __restrict__ y) {
    const int nx = g.nx, ny = g.ny, nz = g.nz, sy = nx;
    const SmLines L(g);
    const int sz = L.P;
    for (int t = threadIdx.x; t < L.P * L.nsplit; t += blockDim.x) {
        const int part = t / L.P, q = t - part * L.P;
        const int j = q / nx, i = q - j * nx;
        const int k0 = part * L.kper, k1 = min(nz, k0 + L.kper);
        if (k0 >= k1) continue;
        int p = q + k0 * sz;
        C xm = k0 > 0 ? x[p - sz] : C(0);
        C x0 = x[p];
        const bool hl = i > 0, hr = i + 1 < nx, hd = j > 0, hu = j + 1 < ny;
        for (int k = k0; k < k1; ++k, p += sz) {
            const C xp = k + 1 < nz ? x[p + sz] : C(0);
            C v;
            if constexpr (sizeof(C) == 8) {
                C nb = xm + xp;
                if (hl) nb += x[p - 1];
                if (hr) nb += x[p + 1];
                if (hd) nb += x[p - sy];
                if (hu) nb += x[p + sy];
                v = fma(b, nb, a * x0);
            } else {
                C d = (x0 - xm) + (x0 - xp);
                d += hl ? x0 - x[p - 1] : x0;
                d += hr ? x0 - x[p + 1] : x0;
                d += hd ? x0 - x[p - sy] : x0;
                d += hu ? x0 - x[p + sy] : x0;
                v = fma(-b, d, (a + C(6) * b) * x0);
            }
            if (z) v = fma(c, z[p], v);
            y[p] = v;
            xm = x0;
            x0 = xp;
        }
    }
    __syncthreads();
}

template <typename C>
__device__ void sm_restrict(const Grid3& gf, const Grid3& gc, const C* __restrict__ f, C* __restrict__ rc) {
    const int nc = gc.n();
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        const int I = q % gc.nx, J = (q / gc.nx) % gc.ny, K = q / (gc.nx * gc.ny);
        const int fi = 2 * I + 1, fj = 2 * J + 1, fk = 2 * K + 1;
        C sacc = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            const int kk = fk + dz;
            if (kk >= gf.nz) continue;
            const C wz = dz == 0 ? C(1) : C(0.5);
            for (int dy = -1; dy <= 1; ++dy) {
                const int jj = fj + dy;
                if (jj >= gf.ny) continue;
                const C wzy = wz * (dy == 0 ? C(1) : C(0.5));
                const int row = gf.nx * (jj + gf.ny * kk);
                C t = f[row + fi];
                if (fi - 1 >= 0) t = fma(C(0.5), f[row + fi - 1], t);
                if (fi + 1 < gf.nx) t = fma(C(0.5), f[row + fi + 1], t);
                sacc = fma(wzy, t, sacc);
            }
        }
        rc[q] = C(0.125) * sacc;
    }
    __syncthreads();
}

// fine index f0 (0-based) -> coarse taps (index, weight) of the trilinear prolongation
__device__ __forceinline__ void sm_taps(int f0, int nc, int& i0, int& i1, float& w0, float& w1) {
    const int f = f0 + 1;
    if ((f & 1) == 0) {
        const int I = f >> 1;
        i0 = I - 1; w0 = I <= nc ? 1.0f : 0.0f;
        i1 = i0;    w1 = 0.0f;
    } else {
        const int I1 = (f - 1) >> 1, I2 = (f + 1) >> 1;
        i0 = I1 - 1; w0 = I1 >= 1 ? 0.5f : 0.0f;
        i1 = I2 - 1; w1 = I2 <= nc ? 0.5f : 0.0f;
    }
    i0 = max(0, min(i0, nc - 1));
    i1 = max(0, min(i1, nc - 1));
}

template <typename C>
__device__ void sm_prolong_add(const Grid3& gf, const Grid3& gc, const C* __restrict__ ec, C* __restrict__ ef) {
    const SmLines L(gf);
    for (int t = threadIdx.x; t < L.P * L.nsplit; t += blockDim.x) {
        const int part = t / L.P, q = t - part * L.P;
        const int j = q / gf.nx, i = q - j * gf.nx;
        const int k0 = part * L.kper, k1 = min(gf.nz, k0 + L.kper);
        int xi[2], yi[2];
        float xw[2], yw[2];
        sm_taps(i, gc.nx, xi[0], xi[1], xw[0], xw[1]);
        sm_taps(j, gc.ny, yi[0], yi[1], yw[0], yw[1]);
        for (int k = k0; k < k1; ++k) {
            int zi[2];
            float zw[2];
            sm_taps(k, gc.nz, zi[0], zi[1], zw[0], zw[1]);
            C sacc = 0;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const C w = C(zw[a]) * C(yw[b]);
                    const int row = gc.nx * (yi[b] + gc.ny * zi[a]);
#pragma unroll
                    for (int d = 0; d < 2; ++d) sacc = fma(w * C(xw[d]), ec[row + xi[d]], sacc);
                }
            ef[q + k * L.P] += sacc;
        }
    }
    __syncthreads();
}

template <typename T, typename C>
__global__ void __launch_bounds__(kSmallThreads)
    k_vcycle_small(SmallLevels L, double omega, int nu_pre, int nu_post, const double* __restrict__ tab,
                   const T* __restrict__ r, int64_t ldr, T* __restrict__ e, int64_t lde) {
    extern __shared__ __align__(16) double smd[];
    const Grid3 gc = L.g[L.nl - 1];
    const int ncs = gc.n();
    const int ntab = gc.nx * gc.nx + gc.ny * gc.ny + gc.nz * gc.nz;
    double* tq = smd;                    // the coarsest level's sine tables Qx, Qy, Qz
    double* u = smd + ntab;              // sine-transform scratch of the coarsest level
    double* v = u + ncs;
    C* sm = reinterpret_cast<C*>(v + ncs);
    const int col = blockIdx.x;
    const int n0 = L.g[0].n();
    C* R0 = sm + L.off[0];
    const double* lam = tab + ntab;      // eigenvalues (global memory; a thread's own one prefetched)
    const bool lam_in_reg = ncs <= (int)blockDim.x;
    const double lam_r = lam_in_reg && (int)threadIdx.x < ncs ? __ldg(lam + threadIdx.x) : 1.0;
    for (int p = threadIdx.x; p < ntab; p += blockDim.x) tq[p] = __ldg(tab + p);
    for (int p = threadIdx.x; p < n0; p += blockDim.x) R0[p] = C(ld_as(r + (int64_t)col * ldr + p));
    __syncthreads();
    C* fin[kFuseMaxLevels];    // final e of each level
    C* oth[kFuseMaxLevels];
    const C w = C(omega);
    for (int l = 0; l < L.nl - 1; ++l) {
        const Grid3 g = L.g[l];
        const int nl = g.n();
        const C s = C(L.s[l]), alpha = C(omega / (6.0 * L.s[l]));
        C* Rl = sm + L.off[l];
        C* c = Rl + nl;
        C* o = Rl + 2 * nl;
        int done;
        if (nu_pre >= 2) { sm_axpby(g, alpha * (C(2) - w), alpha * w / C(6), Rl, C(0), (const C*)nullptr, c); done = 2; }
        else { sm_axpby(g, alpha, C(0), Rl, C(0), (const C*)nullptr, c); done = 1; }
        for (; done < nu_pre; ++done) {
            sm_axpby(g, C(1) - w, w / C(6), c, alpha, Rl, o);
            C* t = c; c = o; o = t;
        }
        sm_axpby(g, -C(6) * s, s, c, C(1), Rl, o);          // residual r - A e
        sm_restrict(g, L.g[l + 1], o, sm + L.off[l + 1]);
        fin[l] = c;
        oth[l] = o;
    }
    {   // coarsest: e = Q diag(1/lambda) Q r
        const C* Rc = sm + L.off[L.nl - 1];
        C* Ec = sm + L.off[L.nl - 1] + ncs;
        const double* Qx = tq;
        const double* Qy = Qx + gc.nx * gc.nx;
        const double* Qz = Qy + gc.ny * gc.ny;
        for (int p = threadIdx.x; p < ncs; p += blockDim.x) u[p] = (double)Rc[p];
        __syncthreads();
        sine_pass_sm(gc, 0, Qx, u, v);
        sine_pass_sm(gc, 1, Qy, v, u);
        sine_pass_sm(gc, 2, Qz, u, v);
        for (int p = threadIdx.x; p < ncs; p += blockDim.x) v[p] /= lam_in_reg ? lam_r : __ldg(lam + p);
        __syncthreads();
        sine_pass_sm(gc, 0, Qx, v, u);
        sine_pass_sm(gc, 1, Qy, u, v);
        sine_pass_sm(gc, 2, Qz, v, u);
        for (int p = threadIdx.x; p < ncs; p += blockDim.x) Ec[p] = C(u[p]);
        __syncthreads();
        fin[L.nl - 1] = Ec;
    }
    for (int l = L.nl - 2; l >= 0; --l) {
        const Grid3 g = L.g[l];
        const C alpha = C(omega / (6.0 * L.s[l]));
        C* Rl = sm + L.off[l];
        C* c = fin[l];
        C* o = oth[l];
        sm_prolong_add(g, L.g[l + 1], fin[l + 1], c);
        for (int k = 0; k < nu_post; ++k) {
            sm_axpby(g, C(1) - w, w / C(6), c, alpha, Rl, o);
            C* t = c; c = o; o = t;
        }
        fin[l] = c;
    }
    for (int p = threadIdx.x; p < n0; p += blockDim.x) st_as(e + (int64_t)col * lde + p, fin[0][p]);
}

template <typename TS, typename TD>
__global__ void k_convert(int64_t n, int ncols, const TS* __restrict__ src, int64_t lds,
                          TD* __restrict__ dst, int64_t ldd) {
    const int64_t total = n * ncols;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / n, p = t - j * n;
        st_as(dst + j * ldd + p, ld_as(src + j * lds + p));
    }
}

template <typename T>
void stencil_t(const Grid3& g, int ncols, double a, double b, const void* x, int64_t ldx, double c,
               const void* z, int64_t ldz, void* y, int64_t ldy, cudaStream_t st) {
    using C = typename Acc<T>::type;
    const int zc = zchunk_for(g.nz);
    const int nzc = (int)ceil_div(g.nz, zc);
    dim3 block(kTX, kTY);
    if constexpr (!std::is_same<T, double>::value) {
        constexpr uintptr_t al = 4 * sizeof(T);    // one 4-point vector
        if (g.nx % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && (!z || ldz % 4 == 0) &&
            ((uintptr_t)x | (uintptr_t)y | (uintptr_t)z) % al == 0) {
            // rows of fewer than 32 vectors: narrower, taller blocks keep every lane busy
            const int nx4 = g.nx / 4;
            const bool four = g.nz >= 64;            // 4-plane runs on large grids, 2-plane runs below
            const int nzc4 = (int)ceil_div(g.nz, four ? 4 : 2);
            const dim3 block4 = nx4 >= 32 ? dim3(32, 4) : (nx4 >= 16 ? dim3(16, 8) : dim3(8, 16));
            dim3 grid4((unsigned)ceil_div(nx4, (int)block4.x), (unsigned)ceil_div(g.ny, (int)block4.y),
                       (unsigned)(nzc4 * ncols));
            const float fa = (float)a, fb = (float)b, fc = (float)c;
            if (z && four)
                k_stencil_v4<T, true, 4><<<grid4, block4, 0, st>>>(g, nzc4, fa, fb, (const T*)x, ldx, fc, (const T*)z, ldz,
                                                                   (T*)y, ldy);
            else if (z)
                k_stencil_v4<T, true, 2><<<grid4, block4, 0, st>>>(g, nzc4, fa, fb, (const T*)x, ldx, fc, (const T*)z, ldz,
                                                                   (T*)y, ldy);
            else if (four)
                k_stencil_v4<T, false, 4><<<grid4, block4, 0, st>>>(g, nzc4, fa, fb, (const T*)x, ldx, 0.f, nullptr, 0,
                                                                    (T*)y, ldy);
            else
                k_stencil_v4<T, false, 2><<<grid4, block4, 0, st>>>(g, nzc4, fa, fb, (const T*)x, ldx, 0.f, nullptr, 0,
                                                                    (T*)y, ldy);
            return;
        }
    }
    dim3 grid((unsigned)ceil_div(g.nx, kTX), (unsigned)ceil_div(g.ny, kTY), (unsigned)(nzc * ncols));
    if (z)
        k_stencil_axpby<T, true><<<grid, block, 0, st>>>(g, zc, nzc, (C)a, (C)b, (const T*)x, ldx, (C)c,
                                                         (const T*)z, ldz, (T*)y, ldy);
    else
        k_stencil_axpby<T, false><<<grid, block, 0, st>>>(g, zc, nzc, (C)a, (C)b, (const T*)x, ldx, C(0),
                                                          nullptr, 0, (T*)y, ldy);
}

template <typename TF, typename TC>
void restrict_t(const Grid3& gf, const Grid3& gc, int ncols, const void* rf, int64_t ldf, void* rc,
                int64_t ldc, cudaStream_t st) {
    if constexpr (!std::is_same<TF, double>::value) {
        constexpr uintptr_t al = 4 * sizeof(TF);
        if (gf.nx % 4 == 0 && ldf % 4 == 0 && (uintptr_t)rf % al == 0) {
            const int kchunk = gc.nz >= 64 ? 8 : (gc.nz >= 16 ? 4 : 2);
            const int nkc = (int)ceil_div(gc.nz, kchunk);
            const int pairs = (int)ceil_div(gc.nx, 2);
            const dim3 block = pairs >= 32 ? dim3(32, 4) : (pairs >= 16 ? dim3(16, 8) : dim3(8, 16));
            dim3 grid((unsigned)ceil_div(pairs, (int)block.x), (unsigned)ceil_div(gc.ny, (int)block.y),
                      (unsigned)(nkc * ncols));
            k_restrict_v4<TF, TC><<<grid, block, 0, st>>>(gf, gc, kchunk, nkc, (const TF*)rf, ldf, (TC*)rc, ldc);
            return;
        }
    }
    dim3 grid((unsigned)ceil_div(gc.nx, kTX), (unsigned)ceil_div(gc.ny, kTY), (unsigned)(gc.nz * ncols));
    k_restrict<TF, TC><<<grid, dim3(kTX, kTY), 0, st>>>(gf, gc, (const TF*)rf, ldf, (TC*)rc, ldc);
}

template <typename TC, typename TF>
void prolong_t(const Grid3& gf, const Grid3& gc, int ncols, const void* ec, int64_t ldc, void* ef, int64_t ldf,
               cudaStream_t st) {
    if constexpr (!std::is_same<TF, double>::value && !std::is_same<TC, double>::value) {
        if (gf.nx % 4 == 0 && ldf % 4 == 0 && ldc % 2 == 0 && (uintptr_t)ef % (4 * sizeof(TF)) == 0 &&
            (uintptr_t)ec % (2 * sizeof(TC)) == 0) {
            const int quads = gf.nx / 4, pairs = (gf.ny + 1) / 2, ncz = (gf.nz + 1) / 2;
            const int zc = ncz >= 64 ? 4 : (ncz >= 8 ? 2 : 1);
            const int nzc = (int)ceil_div(ncz, zc);
            const dim3 block = quads >= 32 ? dim3(32, 4) : (quads >= 16 ? dim3(16, 8) : dim3(8, 16));
            dim3 grid((unsigned)ceil_div(quads, (int)block.x), (unsigned)ceil_div(pairs, (int)block.y),
                      (unsigned)(nzc * ncols));
            k_prolong_v4<TC, TF><<<grid, block, 0, st>>>(gf, gc, zc, nzc, (const TC*)ec, ldc, (TF*)ef, ldf);
            return;
        }
    }
    const int zc = zchunk_for(gc.nz + 1);
    const int nzc = (int)ceil_div(gc.nz + 1, zc);
    dim3 grid((unsigned)ceil_div(gc.nx + 1, kTX), (unsigned)ceil_div(gc.ny + 1, kTY), (unsigned)(nzc * ncols));
    k_prolong_add<TC, TF><<<grid, dim3(kTX, kTY), 0, st>>>(gf, gc, zc, nzc, (const TC*)ec, ldc, (TF*)ef, ldf);
}

template <typename TS, typename TD>
void convert_t(int64_t n, int ncols, const void* src, int64_t lds, void* dst, int64_t ldd, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(ceil_div(n * ncols, 256), (int64_t)kNumSMs * 16);
    k_convert<TS, TD><<<(unsigned)blocks, 256, 0, st>>>(n, ncols, (const TS*)src, lds, (TD*)dst, ldd);
}

}  // namespace

void launch_stencil_axpby(const Grid3& g, int ncols, DType t, double a, double b, const void* x,
                          int64_t ldx, double c, const void* z, int64_t ldz, void* y,
                          int64_t ldy, cudaStream_t st) {
    if (ncols <= 0 || g.n() == 0) return;
    switch (t) {
        case DT_F64: stencil_t<double>(g, ncols, a, b, x, ldx, c, z, ldz, y, ldy, st); break;
        case DT_F32: stencil_t<float>(g, ncols, a, b, x, ldx, c, z, ldz, y, ldy, st); break;
        case DT_BF16: stencil_t<__nv_bfloat16>(g, ncols, a, b, x, ldx, c, z, ldz, y, ldy, st); break;
    }
    LG_CHECK_LAUNCH();
}

void launch_restrict(const Grid3& gf, const Grid3& gc, int ncols, DType tf, const void* rf,
                     int64_t ldf, DType tc, void* rc, int64_t ldc, cudaStream_t st) {
    if (ncols <= 0) return;
    if (tf == DT_F64 && tc == DT_F64) restrict_t<double, double>(gf, gc, ncols, rf, ldf, rc, ldc, st);
    else if (tf == DT_F32 && tc == DT_BF16) restrict_t<float, __nv_bfloat16>(gf, gc, ncols, rf, ldf, rc, ldc, st);
    else if (tf == DT_F32 && tc == DT_F32) restrict_t<float, float>(gf, gc, ncols, rf, ldf, rc, ldc, st);
    else if (tf == DT_BF16 && tc == DT_BF16) restrict_t<__nv_bfloat16, __nv_bfloat16>(gf, gc, ncols, rf, ldf, rc, ldc, st);
    else throw Error(LOBPCG_ERR_ARG, "unsupported restriction types");
    LG_CHECK_LAUNCH();
}

void launch_prolong_add(const Grid3& gf, const Grid3& gc, int ncols, DType tc, const void* ec,
                        int64_t ldc, DType tf, void* ef, int64_t ldf, cudaStream_t st) {
    if (ncols <= 0) return;
    if (tc == DT_F64 && tf == DT_F64) prolong_t<double, double>(gf, gc, ncols, ec, ldc, ef, ldf, st);
    else if (tc == DT_BF16 && tf == DT_F32) prolong_t<__nv_bfloat16, float>(gf, gc, ncols, ec, ldc, ef, ldf, st);
    else if (tc == DT_F32 && tf == DT_F32) prolong_t<float, float>(gf, gc, ncols, ec, ldc, ef, ldf, st);
    else if (tc == DT_BF16 && tf == DT_BF16) prolong_t<__nv_bfloat16, __nv_bfloat16>(gf, gc, ncols, ec, ldc, ef, ldf, st);
    else throw Error(LOBPCG_ERR_ARG, "unsupported prolongation types");
    LG_CHECK_LAUNCH();
}

int64_t coarse_tables_size(const Grid3& g) {
    return (int64_t)g.nx * g.nx + (int64_t)g.ny * g.ny + (int64_t)g.nz * g.nz + g.n();
}

void launch_coarse_setup(const Grid3& g, double scale, double* tables, cudaStream_t st) {
    const int64_t total = coarse_tables_size(g);
    k_coarse_setup<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(g, scale, tables);
    LG_CHECK_LAUNCH();
}

void launch_coarse_solve(const Grid3& g, int ncols, DType t, const double* tables, const void* r,
                         int64_t ldr, void* e, int64_t lde, cudaStream_t st) {
    if (ncols <= 0) return;
    const size_t smem = 2 * (size_t)g.n() * sizeof(double);
    const int maxsmem = 2 * 4096 * (int)sizeof(double);
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    static bool attr_set[64][3] = {};
    if (dev < 64 && !attr_set[dev][t]) {
        if (t == DT_F64) LG_CUDA(cudaFuncSetAttribute(k_coarse_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem));
        if (t == DT_F32) LG_CUDA(cudaFuncSetAttribute(k_coarse_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem));
        if (t == DT_BF16) LG_CUDA(cudaFuncSetAttribute(k_coarse_solve<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsmem));
        attr_set[dev][t] = true;
    }
    switch (t) {
        case DT_F64: k_coarse_solve<double><<<ncols, 256, smem, st>>>(g, tables, (const double*)r, ldr, (double*)e, lde); break;
        case DT_F32: k_coarse_solve<float><<<ncols, 256, smem, st>>>(g, tables, (const float*)r, ldr, (float*)e, lde); break;
        case DT_BF16: k_coarse_solve<__nv_bfloat16><<<ncols, 256, smem, st>>>(g, tables, (const __nv_bfloat16*)r, ldr, (__nv_bfloat16*)e, lde); break;
    }
    LG_CHECK_LAUNCH();
}

void launch_convert(int64_t n, int ncols, DType ts, const void* src, int64_t lds, DType td,
                    void* dst, int64_t ldd, cudaStream_t st) {
    if (ncols <= 0 || n <= 0) return;
    if (ts == DT_F64 && td == DT_F32) convert_t<double, float>(n, ncols, src, lds, dst, ldd, st);
    else if (ts == DT_F32 && td == DT_F64) convert_t<float, double>(n, ncols, src, lds, dst, ldd, st);
    else if (ts == DT_F32 && td == DT_F32) convert_t<float, float>(n, ncols, src, lds, dst, ldd, st);
    else if (ts == DT_F64 && td == DT_F64) convert_t<double, double>(n, ncols, src, lds, dst, ldd, st);
    else throw Error(LOBPCG_ERR_ARG, "unsupported conversion");
    LG_CHECK_LAUNCH();
}


size_t vcycle_small_smem(const Grid3* g, int nl, DType t) {
    const size_t cs = t == DT_F64 ? 8 : 4;
    size_t elems = 0;
    for (int l = 0; l < nl; ++l) elems += 3 * (size_t)g[l].n();
    const Grid3& c = g[nl - 1];
    const size_t q = (size_t)c.nx * c.nx + (size_t)c.ny * c.ny + (size_t)c.nz * c.nz;   // staged sine tables
    return (2 * (size_t)c.n() + q) * sizeof(double) + elems * cs;
}

void launch_vcycle_small(const Grid3* g, const double* scales, int nl, double omega, int nu_pre, int nu_post,
                         const double* tables, int ncols, DType t, const void* r, int64_t ldr, void* e,
                         int64_t lde, cudaStream_t st) {
    LG_REQUIRE(nl >= 1 && nl <= kFuseMaxLevels, LOBPCG_ERR_ARG, "too many fused levels");
    SmallLevels L{};
    L.nl = nl;
    int off = 0;
    for (int l = 0; l < nl; ++l) {
        L.g[l] = g[l];
        L.s[l] = scales[l];
        L.off[l] = off;
        off += 3 * (int)g[l].n();
    }
    const size_t smem = vcycle_small_smem(g, nl, t);
    LG_REQUIRE(smem <= 200 * 1024, LOBPCG_ERR_ARG, "fused V-cycle levels do not fit in shared memory");
    static bool attr[64][3] = {};
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && !attr[dev][t]) {
        if (t == DT_F64) LG_CUDA(cudaFuncSetAttribute(k_vcycle_small<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        if (t == DT_F32) LG_CUDA(cudaFuncSetAttribute(k_vcycle_small<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        if (t == DT_BF16) LG_CUDA(cudaFuncSetAttribute(k_vcycle_small<__nv_bfloat16, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr[dev][t] = true;
    }
    switch (t) {
        case DT_F64: k_vcycle_small<double, double><<<ncols, kSmallThreads, smem, st>>>(L, omega, nu_pre, nu_post, tables, (const double*)r, ldr, (double*)e, lde); break;
        case DT_F32: k_vcycle_small<float, float><<<ncols, kSmallThreads, smem, st>>>(L, omega, nu_pre, nu_post, tables, (const float*)r, ldr, (float*)e, lde); break;
        case DT_BF16: k_vcycle_small<__nv_bfloat16, float><<<ncols, kSmallThreads, smem, st>>>(L, omega, nu_pre, nu_post, tables, (const __nv_bfloat16*)r, ldr, (__nv_bfloat16*)e, lde); break;
    }
    LG_CHECK_LAUNCH();
}
}  // namespace lg
