// Streamed tall-skinny products of the mixed form, Y = S C for float32 column blocks S (n rows,
// a few dozen columns) and a small coefficient matrix C, with the input tiles staged by the
// Tensor Memory Accelerator.
//
// A thread block walks tiles of TP consecutive points (TP = 256 or 128).  Thread 0 keeps a ring
// of shared-memory stages filled with one 2-D TMA copy per input block and tile (mbarrier
// completion); every thread owns 4 consecutive points of a tile (float4 reads of the staged
// columns) and kCG output columns, and writes its outputs straight to global memory with
// float4 stores.  Because every input of a tile is in shared memory before any output of that
// tile is written, the products can run in place.  Four forms:
//   PROJECT   V <- V - [L0 L1] C          (block Gram-Schmidt of the mixed form)
//   APPLY     V <- V Rinv, Rinv upper      (Cholesky orthonormalisation, the orthonormalisations of W and P)
//   GENERAL   V <- [L0 L1 V] K             (the last Gram-Schmidt pass and the Cholesky step in
//                                           one pass: K = [-C Rinv; Rinv])
//   UPDATE    P <- W C_W + P C_P (float32), X <- X C_X + P in double-float, X as hi / lo planes
//             (Ritz update, the Ritz update)
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "tma.cuh"

namespace lg {
namespace {

constexpr int kCG = 4;                  // output columns per thread
constexpr int kMaxThreads = 512;
constexpr int kHeader = 128;
constexpr int kSmemBudget = 100 * 1024;  // two blocks per SM (one 8-warp block per SM left it latency-bound)

enum TsmmMode : int { TS_PROJECT = 0, TS_APPLY = 1, TS_UPDATE = 2, TS_GENERAL = 3 };

struct TsmmArgs {
    CUtensorMap map[4];
    int nblk;
    int coff[4], w[4];      // staged column offset and width of each input block
    int Q;                  // staged columns
    int TP;                 // points per tile
    int nstage;
    int spin;               // polls a stage wait may take before it gives up
    int mode;
    int ncols;              // output columns
    int wl;                 // PROJECT: columns of [L0 L1];  UPDATE: m
    int b, bp;              // UPDATE: widths of W and P
    int cp;                 // row length of the coefficient copies in shared memory (ncols rounded to 4)
    int64_t ld, n;
    float* out0;            // PROJECT / APPLY: V;  UPDATE: Xh
    float* out1;            // UPDATE: Xl
    float* out2;            // UPDATE: P (may be null)
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (ah + al) * (bh + bl) in double-float, al*bl dropped.
__device__ __forceinline__ void df_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);
    float s, d;
    two_sum(hi, p, s, d);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(d, fmaf(ah, bl, fmaf(al, bh, e))));
}

__device__ __forceinline__ float f4(const float4& v, int u) {
    return u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
}

__device__ __forceinline__ void store4(float* col, int64_t p0, int64_t n, const float (&v)[4]) {
    if (p0 + 4 <= n) {
        *reinterpret_cast<float4*>(col + p0) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (p0 + u < n) col[p0 + u] = v[u];
    }
}

__global__ void __launch_bounds__(kMaxThreads)
    k_tsmm(const __grid_constant__ TsmmArgs a, const double* __restrict__ C, int ldc,
           const unsigned* __restrict__ status, unsigned skip, unsigned* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (status && (*status & skip)) return;
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    float* stages = reinterpret_cast<float*>(smem + kHeader);
    const int64_t stage_floats = (int64_t)a.Q * a.TP;
    float* coef = stages + a.nstage * stage_floats;     // coefficient copies (float32)
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    // coefficients: [row i][col c] with row length cp; UPDATE: C_X hi, C_X lo, C_W, C_P
    const int cp = a.cp;
    const int crows = a.mode == TS_UPDATE ? 2 * a.wl + a.b + a.bp
                                          : (a.mode == TS_PROJECT ? a.wl : (a.mode == TS_GENERAL ? a.Q : a.ncols));
    for (int e = tid; e < crows * cp; e += nthr) {
        const int i = e / cp, c = e - i * cp;
        float v = 0.f;
        if (c < a.ncols) {
            if (a.mode == TS_UPDATE) {
                const int m = a.wl;
                if (i < m) {
                    v = (float)C[i + (int64_t)ldc * c];
                } else if (i < 2 * m) {
                    const double x = C[(i - m) + (int64_t)ldc * c];
                    v = (float)(x - (double)(float)x);
                } else {
                    v = (float)C[(i - m) + (int64_t)ldc * c];     // C_W rows m.., C_P rows m+b..
                }
            } else if (a.mode == TS_APPLY) {
                v = i <= c ? (float)C[i + (int64_t)ldc * c] : 0.f;
            } else {
                v = (float)C[i + (int64_t)ldc * c];
            }
        }
        coef[e] = v;
    }
    unsigned tx = 0;
    for (int b = 0; b < a.nblk; ++b) tx += (unsigned)(a.TP * a.w[b] * 4);
    const int64_t ntiles = (a.n + a.TP - 1) / a.TP;
    const int mine = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int it) {
        const int buf = it % a.nstage;
        const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
        float* dst = stages + buf * stage_floats;
        mbar_expect_tx(&full[buf], tx);
        for (int b = 0; b < a.nblk; ++b)
            tma_load_2d(dst + (int64_t)a.coff[b] * a.TP, &a.map[b], (int)(tile * a.TP), 0, &full[buf]);
    };
    if (tid == 0)
        for (int it = 0; it < min(mine, a.nstage); ++it) issue(it);

    const int lanes = a.TP / 4;
    const int pl = tid % lanes;                 // point group: points 4 pl .. 4 pl + 3 of the tile
    const int c0 = (tid / lanes) * kCG;         // first output column
    const bool active = c0 < a.ncols;
    for (int it = 0; it < mine; ++it) {
        const int buf = it % a.nstage;
        const bool ok = mbar_wait(&full[buf], (unsigned)((it / a.nstage) & 1), a.spin);
        const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
        const int64_t p0 = tile * a.TP + 4 * pl;
        if (ok && active && p0 < a.n) {
            const float* sm = stages + buf * stage_floats + 4 * pl;
            if (a.mode == TS_UPDATE) {
                const int m = a.wl;
                float ph[4][kCG], xh[4][kCG], xl[4][kCG];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < kCG; ++v) ph[u][v] = xh[u][v] = xl[u][v] = 0.f;
                const float* cxh = coef;
                const float* cxl = coef + m * cp;
                const float* cwp = coef + 2 * m * cp;          // C_W then C_P rows
                const int nwp = a.b + a.bp;
                const int wcol = a.coff[2];                    // staged W then P columns
                for (int i = 0; i < nwp; ++i) {
                    const float4 s = *reinterpret_cast<const float4*>(sm + (int64_t)(wcol + i) * a.TP);
                    const float4 cc = *reinterpret_cast<const float4*>(cwp + i * cp + c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float su = f4(s, u);
                        ph[u][0] = fmaf(su, cc.x, ph[u][0]);
                        ph[u][1] = fmaf(su, cc.y, ph[u][1]);
                        ph[u][2] = fmaf(su, cc.z, ph[u][2]);
                        ph[u][3] = fmaf(su, cc.w, ph[u][3]);
                    }
                }
                for (int i = 0; i < m; ++i) {
                    const float4 ah = *reinterpret_cast<const float4*>(sm + (int64_t)i * a.TP);
                    const float4 al = *reinterpret_cast<const float4*>(sm + (int64_t)(a.coff[1] + i) * a.TP);
                    const float4 bh = *reinterpret_cast<const float4*>(cxh + i * cp + c0);
                    const float4 bl = *reinterpret_cast<const float4*>(cxl + i * cp + c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float h = f4(ah, u), l = f4(al, u);
                        df_mac(xh[u][0], xl[u][0], h, l, bh.x, bl.x);
                        df_mac(xh[u][1], xl[u][1], h, l, bh.y, bl.y);
                        df_mac(xh[u][2], xl[u][2], h, l, bh.z, bl.z);
                        df_mac(xh[u][3], xl[u][3], h, l, bh.w, bl.w);
                    }
                }
#pragma unroll
                for (int v = 0; v < kCG; ++v) {
                    const int c = c0 + v;
                    if (c >= a.ncols) break;
                    float oh[4], ol[4], op[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float s, e;
                        two_sum(xh[u][v], ph[u][v], s, e);     // X C_X + P
                        const float l = __fadd_rn(xl[u][v], e);
                        oh[u] = __fadd_rn(s, l);
                        ol[u] = __fsub_rn(l, __fsub_rn(oh[u], s));
                        op[u] = ph[u][v];
                    }
                    store4(a.out0 + (int64_t)c * a.ld, p0, a.n, oh);
                    store4(a.out1 + (int64_t)c * a.ld, p0, a.n, ol);
                    if (a.out2) store4(a.out2 + (int64_t)c * a.ld, p0, a.n, op);
                }
            } else {
                float acc[4][kCG];
                const int vcol = a.mode == TS_PROJECT ? a.coff[a.nblk - 1] : 0;   // staged V
#pragma unroll
                for (int v = 0; v < kCG; ++v) {
                    const int c = min(c0 + v, a.ncols - 1);
                    const float4 x = a.mode == TS_PROJECT
                                         ? *reinterpret_cast<const float4*>(sm + (int64_t)(vcol + c) * a.TP)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[u][v] = f4(x, u);
                }
                // PROJECT: the [L0 L1] columns are staged first; APPLY: V itself (rows i <= c);
                // GENERAL: every staged column
                const int nin = a.mode == TS_PROJECT ? a.wl : (a.mode == TS_GENERAL ? a.Q : min(a.ncols, c0 + kCG));
                const float sg = a.mode == TS_PROJECT ? -1.f : 1.f;
                for (int i = 0; i < nin; ++i) {
                    const float4 s = *reinterpret_cast<const float4*>(sm + (int64_t)i * a.TP);
                    const float4 cc = *reinterpret_cast<const float4*>(coef + i * cp + c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float su = sg * f4(s, u);
                        acc[u][0] = fmaf(su, cc.x, acc[u][0]);
                        acc[u][1] = fmaf(su, cc.y, acc[u][1]);
                        acc[u][2] = fmaf(su, cc.z, acc[u][2]);
                        acc[u][3] = fmaf(su, cc.w, acc[u][3]);
                    }
                }
#pragma unroll
                for (int v = 0; v < kCG; ++v) {
                    const int c = c0 + v;
                    if (c >= a.ncols) break;
                    const float o[4] = {acc[0][v], acc[1][v], acc[2][v], acc[3][v]};
                    store4(a.out0 + (int64_t)c * a.ld, p0, a.n, o);
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(err, ST_TIMEOUT);
                // the stages issued from `it` on may still be in flight; one budget of polls
                int budget = kSpinLimit;
                for (int j = it; j < min(mine, it + a.nstage); ++j)
                    (void)mbar_wait_budget(&full[j % a.nstage], (unsigned)((j / a.nstage) & 1), budget);
            }
            return;
        }
        if (tid == 0 && it + a.nstage < mine) issue(it + a.nstage);
    }
}

struct TsBlock {
    const float* p;
    int w;
};

void tsmm_launch(TsmmArgs& a, const TsBlock* blk, int nblk, const double* C, int ldc, const unsigned* status,
                 unsigned skip, unsigned* err, cudaStream_t st) {
    a.nblk = 0;
    int off = 0;
    for (int b = 0; b < nblk; ++b) {
        a.coff[b] = off;          // kept for every listed block (zero-width ones too)
        a.w[b] = blk[b].w;
        off += blk[b].w;
    }
    a.Q = off;
    // TP: 256 points if three stages fit, else 128
    a.TP = 256;
    while (a.TP > 64 && 3 * (int64_t)a.Q * a.TP * 4 > kSmemBudget) a.TP /= 2;
    const int64_t stage_bytes = (int64_t)a.Q * a.TP * 4;
    const int crows = a.mode == TS_UPDATE ? 2 * a.wl + a.b + a.bp
                                          : (a.mode == TS_PROJECT ? a.wl : (a.mode == TS_GENERAL ? a.Q : a.ncols));
    a.cp = (a.ncols + 3) & ~3;
    const int64_t coef_bytes = (int64_t)crows * a.cp * 4;
    a.nstage = (int)std::max<int64_t>(2, std::min<int64_t>(4, (kSmemBudget - coef_bytes) / stage_bytes));
    a.spin = stage_wait_polls();
    const size_t smem = 2 * kHeader + a.nstage * stage_bytes + coef_bytes;
    LG_REQUIRE(smem <= 227 * 1024, LOBPCG_ERR_ARG, "streamed product does not fit in shared memory");
    // tensor maps of the non-empty blocks, in the order of their staged offsets
    int k = 0;
    for (int b = 0; b < nblk; ++b) {
        if (blk[b].w <= 0) continue;
        encode_f32_cols(&a.map[k], blk[b].p, a.n, blk[b].w, a.ld, a.TP);
        a.coff[k] = a.coff[b];
        a.w[k] = a.w[b];
        ++k;
    }
    a.nblk = k;
    const int threads = (a.TP / 4) * (int)ceil_div(a.ncols, kCG);
    LG_REQUIRE(threads <= kMaxThreads, LOBPCG_ERR_ARG, "too many output columns for the streamed product");
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        LG_CUDA(cudaFuncSetAttribute(k_tsmm, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set.fetch_or(bit);
    }
    const int64_t ntiles = ceil_div(a.n, a.TP);
    const int per_sm = std::max(1, (int)((227 * 1024) / smem));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)kNumSMs * per_sm));
    k_tsmm<<<(unsigned)grid, threads, smem, st>>>(a, C, ldc, status, skip, err);
    LG_CHECK_LAUNCH();
}

}  // namespace

void launch_project32(int64_t n, int b, float* V, const float* L0, int w0, const float* L1, int w1, int64_t ld,
                      const double* C, int ldc, unsigned* err, cudaStream_t st) {
    if (b <= 0 || w0 + w1 <= 0) return;
    static thread_local TsmmArgs a;
    a = TsmmArgs{};
    a.mode = TS_PROJECT;
    a.ncols = b;
    a.wl = w0 + w1;
    a.ld = ld;
    a.n = n;
    a.out0 = V;
    const TsBlock blk[3] = {{L0, w0}, {L1, w1}, {V, b}};
    tsmm_launch(a, blk, 3, C, ldc, nullptr, 0u, err, st);
}

void launch_combine32(int64_t n, int b, float* V, const float* L0, int w0, const float* L1, int w1, int64_t ld,
                      const double* K, int ldk, const unsigned* status, unsigned skip, unsigned* err,
                      cudaStream_t st) {
    if (b <= 0) return;
    static thread_local TsmmArgs a;
    a = TsmmArgs{};
    a.mode = TS_GENERAL;
    a.ncols = b;
    a.wl = w0 + w1;
    a.ld = ld;
    a.n = n;
    a.out0 = V;
    const TsBlock blk[3] = {{L0, w0}, {L1, w1}, {V, b}};
    tsmm_launch(a, blk, 3, K, ldk, status, skip, err, st);
}

void launch_apply32(int64_t n, int b, float* V, int64_t ld, const double* Rinv, const unsigned* status,
                    unsigned skip, unsigned* err, cudaStream_t st) {
    if (b <= 0) return;
    static thread_local TsmmArgs a;
    a = TsmmArgs{};
    a.mode = TS_APPLY;
    a.ncols = b;
    a.ld = ld;
    a.n = n;
    a.out0 = V;
    const TsBlock blk[1] = {{V, b}};
    tsmm_launch(a, blk, 1, Rinv, b, status, skip, err, st);
}

void launch_update_mx2(int64_t n, int m, float* Xh, float* Xl, const float* W, int b, const float* P, int bp,
                       int64_t ld, const double* C, int q, float* Pout, const unsigned* status, unsigned skip,
                       unsigned* err, cudaStream_t st) {
    static thread_local TsmmArgs a;
    a = TsmmArgs{};
    a.mode = TS_UPDATE;
    a.ncols = m;
    a.wl = m;
    a.b = b;
    a.bp = bp;
    a.ld = ld;
    a.n = n;
    a.out0 = Xh;
    a.out1 = Xl;
    a.out2 = Pout;
    const TsBlock blk[4] = {{Xh, m}, {Xl, m}, {W, b}, {P, bp}};
    tsmm_launch(a, blk, 4, C, q, status, skip, err, st);
}

}  // namespace lg
