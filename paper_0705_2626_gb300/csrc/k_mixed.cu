// Kernels of the mixed form that keep X in double-float arithmetic on the float32 pipe (the
// double-float Ritz update is the UPDATE form of k_tsmm.cu).
//
// In the mixed form the Ritz vectors X live in two float32 planes, X = Xh + Xl (about 48
// significant bits, 2^-48 relative -- well below what the 1e-8 residual tolerance needs), so that
// the two X-side operations of every iteration run on the float32 units instead of GB300's
// float64 units (1/64 of the float32 rate):
//   * the Ritz update (Section 2.2; k_tsmm.cu);
//   * the residual (the residuals) R = A X - X Lambda from the planes, with the 7-point stencil and the
//     Lambda X product in double-float and R rounded to float32 at the end, plus the squared
//     column norms.
// Double-float conventions: a product a*b of float32 values is made exact as (p, e) with
// p = fl(a*b), e = fma(a, b, -p); sums of two floats are made exact with Knuth's two-sum.  The
// _rn intrinsics keep the compiler from contracting a multiply into a following add.
#include <algorithm>

#include "common.cuh"

namespace lg {
namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void split(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

constexpr int kTX = 32, kTY = 4;

__host__ __device__ inline int zchunk_mx(int nz) { return nz >= 64 ? 16 : (nz >= 16 ? 8 : nz); }

// R[:, j] = A X[:, j] - lambda_j X[:, j] from the planes; partial[j * nblk + block] = sum r^2
// over the block's points.  A = scale * (6 I - sum of the 6 neighbours), zero outside the grid.
// Each thread owns an (i, j) line and marches along k through a chunk of planes.
__global__ void __launch_bounds__(kTX* kTY)
    k_resid_mx(Grid3 g, int zchunk, int nzc, double scale, const float* __restrict__ Xh,
               const float* __restrict__ Xl, int64_t ld, const double* __restrict__ lam, float* __restrict__ R,
               int64_t ldr, double* __restrict__ partial) {
    const int i = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    const int nblk = gridDim.x * gridDim.y * nzc;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * kc);
    float sh, sl, lh, ll;
    split(scale, sh, sl);
    split(lam[col], lh, ll);
    float acc = 0.f;
    if (i < g.nx && j < g.ny) {
        const int k0 = kc * zchunk;
        const int k1 = min(k0 + zchunk, g.nz);
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        const float* xh = Xh + (int64_t)col * ld;
        const float* xl = Xl + (int64_t)col * ld;
        float* rc = R + (int64_t)col * ldr;
        int64_t p = i + sy * (j + (int64_t)g.ny * k0);
        float mh = 0.f, ml = 0.f;
        if (k0 > 0) { mh = __ldg(xh + p - sz); ml = __ldg(xl + p - sz); }
        float ch = __ldg(xh + p), cl = __ldg(xl + p);
        const bool hl = i > 0, hr = i + 1 < g.nx, hd = j > 0, hu = j + 1 < g.ny;
        for (int k = k0; k < k1; ++k, p += sz) {
            float ph = 0.f, pl = 0.f;
            if (k + 1 < g.nz) { ph = __ldg(xh + p + sz); pl = __ldg(xl + p + sz); }
            // y = 6 x_p - sum_q x_q
            float hi = __fmul_rn(6.f, ch);
            float lo = fmaf(6.f, cl, fmaf(6.f, ch, -hi));
            auto sub = [&](float qh, float ql) {
                float s, e;
                two_sum(hi, -qh, s, e);
                hi = s;
                lo = __fsub_rn(__fadd_rn(lo, e), ql);
            };
            sub(mh, ml);
            sub(ph, pl);
            if (hl) sub(__ldg(xh + p - 1), __ldg(xl + p - 1));
            if (hr) sub(__ldg(xh + p + 1), __ldg(xl + p + 1));
            if (hd) sub(__ldg(xh + p - sy), __ldg(xl + p - sy));
            if (hu) sub(__ldg(xh + p + sy), __ldg(xl + p + sy));
            // scale * y and lambda * x, then their difference
            const float yh = __fmul_rn(hi, sh);
            const float ye = fmaf(lo, sh, fmaf(hi, sl, fmaf(hi, sh, -yh)));
            const float qh = __fmul_rn(lh, ch);
            const float qe = fmaf(ll, ch, fmaf(lh, cl, fmaf(lh, ch, -qh)));
            float s, e;
            two_sum(yh, -qh, s, e);
            const float r = __fadd_rn(s, __fadd_rn(e, __fsub_rn(ye, qe)));
            rc[p] = r;
            acc = fmaf(r, r, acc);
            mh = ch; ml = cl;
            ch = ph; cl = pl;
        }
    }
    // block sum of the float32 per-thread sums (at most zchunk terms each), in float64
    double v = acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = threadIdx.y * kTX + threadIdx.x;
    __shared__ double redd[kTX * kTY / 32];
    if ((t & 31) == 0) redd[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kTX * kTY / 32; ++w) s += redd[w];
        partial[(int64_t)col * nblk + bid] = s;
    }
}

// The same residual for nx divisible by 4: each thread owns 4 consecutive points of an x-row
// (float4 loads of both planes); identical arithmetic per point.
__global__ void __launch_bounds__(kTX* kTY)
    k_resid_mx4(Grid3 g, int zchunk, int nzc, double scale, const float* __restrict__ Xh,
                const float* __restrict__ Xl, int64_t ld, const double* __restrict__ lam, float* __restrict__ R,
                int64_t ldr, double* __restrict__ partial) {
    const int i4 = blockIdx.x * kTX + threadIdx.x;
    const int j = blockIdx.y * kTY + threadIdx.y;
    const int col = blockIdx.z / nzc;
    const int kc = blockIdx.z - col * nzc;
    const int nblk = gridDim.x * gridDim.y * nzc;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * kc);
    float sh, sl, lh, ll;
    split(scale, sh, sl);
    split(lam[col], lh, ll);
    float acc = 0.f;
    if (4 * i4 < g.nx && j < g.ny) {
        const int i0 = 4 * i4;
        const int k0 = kc * zchunk;
        const int k1 = min(k0 + zchunk, g.nz);
        const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
        const float* xh = Xh + (int64_t)col * ld;
        const float* xl = Xl + (int64_t)col * ld;
        float* rc = R + (int64_t)col * ldr;
        auto l4 = [](const float* q) { return __ldg(reinterpret_cast<const float4*>(q)); };
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t p = i0 + sy * (j + (int64_t)g.ny * k0);
        float4 mh = z4, ml = z4;
        if (k0 > 0) { mh = l4(xh + p - sz); ml = l4(xl + p - sz); }
        float4 ch = l4(xh + p), cl = l4(xl + p);
        const bool hl = i0 > 0, hr = i0 + 4 < g.nx, hd = j > 0, hu = j + 1 < g.ny;
        for (int k = k0; k < k1; ++k, p += sz) {
            float4 ph = z4, pl = z4;
            if (k + 1 < g.nz) { ph = l4(xh + p + sz); pl = l4(xl + p + sz); }
            const float4 dh = hd ? l4(xh + p - sy) : z4, dl = hd ? l4(xl + p - sy) : z4;
            const float4 uh = hu ? l4(xh + p + sy) : z4, ul = hu ? l4(xl + p + sy) : z4;
            const float lfh = hl ? __ldg(xh + p - 1) : 0.f, lfl = hl ? __ldg(xl + p - 1) : 0.f;
            const float rth = hr ? __ldg(xh + p + 4) : 0.f, rtl = hr ? __ldg(xl + p + 4) : 0.f;
            const float chv[6] = {lfh, ch.x, ch.y, ch.z, ch.w, rth};
            const float clv[6] = {lfl, cl.x, cl.y, cl.z, cl.w, rtl};
            const float mhv[4] = {mh.x, mh.y, mh.z, mh.w}, mlv[4] = {ml.x, ml.y, ml.z, ml.w};
            const float phv[4] = {ph.x, ph.y, ph.z, ph.w}, plv[4] = {pl.x, pl.y, pl.z, pl.w};
            const float dhv[4] = {dh.x, dh.y, dh.z, dh.w}, dlv[4] = {dl.x, dl.y, dl.z, dl.w};
            const float uhv[4] = {uh.x, uh.y, uh.z, uh.w}, ulv[4] = {ul.x, ul.y, ul.z, ul.w};
            float out[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float xh0 = chv[e + 1], xl0 = clv[e + 1];
                float hi = __fmul_rn(6.f, xh0);
                float lo = fmaf(6.f, xl0, fmaf(6.f, xh0, -hi));
                auto sub = [&](float qh, float ql) {
                    float s, er;
                    two_sum(hi, -qh, s, er);
                    hi = s;
                    lo = __fsub_rn(__fadd_rn(lo, er), ql);
                };
                sub(mhv[e], mlv[e]);
                sub(phv[e], plv[e]);
                sub(chv[e], clv[e]);            // x-1 (zero outside)
                sub(chv[e + 2], clv[e + 2]);    // x+1
                sub(dhv[e], dlv[e]);
                sub(uhv[e], ulv[e]);
                const float yh = __fmul_rn(hi, sh);
                const float ye = fmaf(lo, sh, fmaf(hi, sl, fmaf(hi, sh, -yh)));
                const float qh = __fmul_rn(lh, xh0);
                const float qe = fmaf(ll, xh0, fmaf(lh, xl0, fmaf(lh, xh0, -qh)));
                float s, er;
                two_sum(yh, -qh, s, er);
                const float r = __fadd_rn(s, __fadd_rn(er, __fsub_rn(ye, qe)));
                out[e] = r;
                acc = fmaf(r, r, acc);
            }
            *reinterpret_cast<float4*>(rc + p) = make_float4(out[0], out[1], out[2], out[3]);
            mh = ch; ml = cl;
            ch = ph; cl = pl;
        }
    }
    double v = acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = threadIdx.y * kTX + threadIdx.x;
    __shared__ double redd[kTX * kTY / 32];
    if ((t & 31) == 0) redd[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double sacc = 0.0;
        for (int w = 0; w < kTX * kTY / 32; ++w) sacc += redd[w];
        partial[(int64_t)col * nblk + bid] = sacc;
    }
}

__global__ void k_planes_to_f64(int64_t n, int m, const float* __restrict__ Xh, const float* __restrict__ Xl,
                                int64_t ld, double* __restrict__ X, int64_t ldx) {
    const int c = blockIdx.y;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        X[(int64_t)c * ldx + p] = (double)__ldg(Xh + (int64_t)c * ld + p) + (double)__ldg(Xl + (int64_t)c * ld + p);
}

}  // namespace

static bool resid_vec4(const Grid3& g) { return g.nx % 4 == 0; }

int resid_mx_blocks(const Grid3& g) {
    const int zc = zchunk_mx(g.nz);
    const int64_t gx = resid_vec4(g) ? ceil_div(g.nx / 4, kTX) : ceil_div(g.nx, kTX);
    return (int)(gx * ceil_div(g.ny, kTY) * ceil_div(g.nz, zc));
}

void launch_resid_mx(const Grid3& g, int m, double scale, const float* Xh, const float* Xl, int64_t ld,
                     const double* lam, float* R, int64_t ldr, double* partial, cudaStream_t st) {
    const int zc = zchunk_mx(g.nz);
    const int nzc = (int)ceil_div(g.nz, zc);
    if (resid_vec4(g) && ld % 4 == 0 && ldr % 4 == 0) {
        dim3 grid((unsigned)ceil_div(g.nx / 4, kTX), (unsigned)ceil_div(g.ny, kTY), (unsigned)(nzc * m));
        k_resid_mx4<<<grid, dim3(kTX, kTY), 0, st>>>(g, zc, nzc, scale, Xh, Xl, ld, lam, R, ldr, partial);
    } else {
        dim3 grid((unsigned)ceil_div(g.nx, kTX), (unsigned)ceil_div(g.ny, kTY), (unsigned)(nzc * m));
        k_resid_mx<<<grid, dim3(kTX, kTY), 0, st>>>(g, zc, nzc, scale, Xh, Xl, ld, lam, R, ldr, partial);
    }
    LG_CHECK_LAUNCH();
}

void launch_planes_to_f64(int64_t n, int m, const float* Xh, const float* Xl, int64_t ld, double* X, int64_t ldx,
                          cudaStream_t st) {
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(n, 256), 1024), (unsigned)m);
    k_planes_to_f64<<<grid, 256, 0, st>>>(n, m, Xh, Xl, ld, X, ldx);
    LG_CHECK_LAUNCH();
}

}  // namespace lg
