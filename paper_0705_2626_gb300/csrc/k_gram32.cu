// Tall-skinny Gram products of the mixed form (Section 2.2, on float32
// data), staged into shared memory by the Tensor Memory Accelerator.
//
// Every product here is S_i^T S_j over n grid points for float32 column blocks with a common
// leading dimension.  A thread block owns a contiguous chunk of rows and walks it in stages of K
// rows: one thread issues one 2-D TMA copy (cp.async.bulk.tensor) per column block and stage into
// a ring of shared-memory buffers guarded by mbarriers, so that the next stages stream in while
// the current one is consumed.  In shared memory each column of a stage is K contiguous floats.
// The output is cut into register tiles; `ks` consecutive lanes share a tile and split the rows
// of a stage between them (lane g takes rows 4g, 4g+1, ... in float4 steps), which keeps every
// shared-memory read conflict-free.  At the end the ks lanes are added in a fixed order and
// lane 0 writes the chunk's partial sums (float64); a separate kernel adds the chunks in a
// fixed order, so results are deterministic.
//
// Two arithmetics:
//  * float32 tiles (4 x 8 outputs per thread): float32 products summed in float32 for at
//    least 32 rows per thread, then added into a Kahan-compensated float32 total;
//  * double-float tiles (4 x 4 outputs per thread) for X^T X with X held as float32 hi / lo
//    planes: hi*hi products made exact with an FMA, the hi*lo cross terms added, the sum kept
//    as an unevaluated pair (hi, lo) updated by Knuth's two-sum -- about 2^-44 relative.
//    These are written with the _rn intrinsics so that no multiply is contracted into an add.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "gram_out.cuh"
#include "tma.cuh"

namespace lg {
namespace {

constexpr int kG32Threads = 256;
constexpr int kG32MaxBlocks = 6;
constexpr int kG32MaxTiles = 640;
constexpr int kG32SmemBudget = 200 * 1024;
constexpr int kG32Header = 128;               // mbarriers in front of the stage buffers

struct G32Args {
    CUtensorMap map[kG32MaxBlocks];
    int nblk;
    int coff[kG32MaxBlocks];    // first staged column of each block
    int w[kG32MaxBlocks];
    int Q;                      // staged columns per stage
    int K;                      // rows per stage
    int ks;                     // lanes per tile
    int nstage;                 // depth of the buffer ring
    int spin;                   // polls a stage wait may take before it gives up
    int loff;                   // double-float tiles: staged offset of the lo plane
    int ntiles, tpc, ngroups;   // tiles, tiles per block, blocks per chunk
    int64_t rows_per_chunk, part_stride;
    int nout;
    G32Out out[2];
    uint16_t ti[kG32MaxTiles], tj[kG32MaxTiles];
    uint8_t to[kG32MaxTiles];
};

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// hi/lo += a*b with a = (ah, al), b = (bh, bl); the al*bl term is dropped.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = __fadd_rn(hi, p);
    const float z = __fsub_rn(t, hi);
    const float d = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(d, e));
}

template <bool DF>
struct TileShape;
template <>
struct TileShape<false> { static constexpr int TI = 4, TJ = 8; };
template <>
struct TileShape<true> { static constexpr int TI = 4, TJ = 4; };

template <bool DF>
__global__ void __launch_bounds__(kG32Threads, DF ? 1 : 2)
    k_gram32(const __grid_constant__ G32Args a, int64_t n, double* __restrict__ part, unsigned* status) {
    constexpr int TI = TileShape<DF>::TI, TJ = TileShape<DF>::TJ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned: align the window by hand (kG32Header spare bytes)
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    float* stages = reinterpret_cast<float*>(smem + kG32Header);
    const int64_t stage_floats = (int64_t)a.Q * a.K;
    const int chunk = blockIdx.x / a.ngroups, group = blockIdx.x - chunk * a.ngroups;
    const int64_t r0 = chunk * a.rows_per_chunk;
    const int64_t r1 = min(n, r0 + a.rows_per_chunk);
    const int nst = r1 > r0 ? (int)((r1 - r0 + a.K - 1) / a.K) : 0;
    const int tid = threadIdx.x;
    const int tl = tid / a.ks, kg = tid - tl * a.ks;
    const int tile = group * a.tpc + tl;
    const bool active = tl < a.tpc && tile < a.ntiles;
    const int i0 = active ? a.ti[tile] : 0;
    const int j0 = active ? a.tj[tile] : 0;
    unsigned tx = 0;
    for (int b = 0; b < a.nblk; ++b) tx += (unsigned)(a.K * a.w[b] * 4);

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int st) {
        const int buf = st % a.nstage;
        float* dst = stages + buf * stage_floats;
        mbar_expect_tx(&full[buf], tx);
        for (int b = 0; b < a.nblk; ++b)
            tma_load_2d(dst + (int64_t)a.coff[b] * a.K, &a.map[b], (int)(r0 + (int64_t)st * a.K), 0, &full[buf]);
    };
    if (tid == 0)
        for (int st = 0; st < min(nst, a.nstage); ++st) issue(st);

    // float32 tiles: acc = the current run's sums, tot = Kahan total, cmpb = its compensation
    // kept as bfloat16 pairs (the compensation is ~eps32 |tot|; rounding it to 8 bits changes the
    // total by ~2^-9 eps32 |tot| per flush, and halves its registers so that two blocks fit per
    // SM).  Double-float tiles: tot / cmp = hi / lo of the running sums.
    float acc[TI][TJ], tot[TI][TJ], cmp[TI][TJ];
    __nv_bfloat162 cmpb[TI][TJ / 2];
#pragma unroll
    for (int u = 0; u < TI; ++u) {
#pragma unroll
        for (int v = 0; v < TJ; ++v) acc[u][v] = tot[u][v] = cmp[u][v] = 0.f;
#pragma unroll
        for (int v = 0; v < TJ / 2; ++v) cmpb[u][v] = __floats2bfloat162_rn(0.f, 0.f);
    }

    const int steps = a.K / (4 * a.ks);                       // float4 steps per lane and stage
    const int flush_every = max(1, (32 * a.ks) / a.K);        // >= 32 rows per float32 run
    int failed_at = -1;
    for (int st = 0; st < nst; ++st) {
        const int buf = st % a.nstage;
        const bool ok = mbar_wait(&full[buf], (unsigned)((st / a.nstage) & 1), a.spin);
        if (ok && active) {
            const float* sm = stages + buf * stage_floats;
            for (int s = 0; s < steps; ++s) {
                const int r = 4 * (kg + a.ks * s);
                if constexpr (!DF) {
                    float4 x[TI];
#pragma unroll
                    for (int u = 0; u < TI; ++u) x[u] = lds4(sm + (i0 + u) * a.K + r);
#pragma unroll
                    for (int h = 0; h < TJ / 4; ++h) {
                        float4 y[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) y[v] = lds4(sm + (j0 + 4 * h + v) * a.K + r);
#pragma unroll
                        for (int u = 0; u < TI; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                float t = acc[u][4 * h + v];
                                t = fmaf(x[u].x, y[v].x, t);
                                t = fmaf(x[u].y, y[v].y, t);
                                t = fmaf(x[u].z, y[v].z, t);
                                t = fmaf(x[u].w, y[v].w, t);
                                acc[u][4 * h + v] = t;
                            }
                    }
                } else {
                    float4 xh[TI], xl[TI];
#pragma unroll
                    for (int u = 0; u < TI; ++u) {
                        xh[u] = lds4(sm + (i0 + u) * a.K + r);
                        xl[u] = lds4(sm + (i0 + a.loff + u) * a.K + r);
                    }
#pragma unroll
                    for (int v = 0; v < TJ; ++v) {
                        const float4 yh = lds4(sm + (j0 + v) * a.K + r);
                        const float4 yl = lds4(sm + (j0 + a.loff + v) * a.K + r);
#pragma unroll
                        for (int u = 0; u < TI; ++u) {
                            df_fma(tot[u][v], cmp[u][v], xh[u].x, xl[u].x, yh.x, yl.x);
                            df_fma(tot[u][v], cmp[u][v], xh[u].y, xl[u].y, yh.y, yl.y);
                            df_fma(tot[u][v], cmp[u][v], xh[u].z, xl[u].z, yh.z, yl.z);
                            df_fma(tot[u][v], cmp[u][v], xh[u].w, xl[u].w, yh.w, yl.w);
                        }
                    }
                }
            }
            if constexpr (!DF) {
                if ((st + 1) % flush_every == 0 || st + 1 == nst) {
#pragma unroll
                    for (int u = 0; u < TI; ++u)
#pragma unroll
                        for (int v = 0; v < TJ; v += 2) {
                            float c2[2] = {__low2float(cmpb[u][v / 2]), __high2float(cmpb[u][v / 2])};
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const float y = __fsub_rn(acc[u][v + e], c2[e]);
                                const float t = __fadd_rn(tot[u][v + e], y);
                                c2[e] = __fsub_rn(__fsub_rn(t, tot[u][v + e]), y);
                                tot[u][v + e] = t;
                                acc[u][v + e] = 0.f;
                            }
                            cmpb[u][v / 2] = __floats2bfloat162_rn(c2[0], c2[1]);
                        }
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            failed_at = st;
            break;
        }
        if (tid == 0 && st + a.nstage < nst) issue(st + a.nstage);
    }
    if (failed_at >= 0) {
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            // Stages before failed_at were consumed; those issued after it -- up to failed_at +
            // nstage - 1 -- may still be in flight and must land before the block exits.  One
            // budget of polls bounds the whole clean-up.
            int budget = kSpinLimit;
            const int issued_end = min(nst, failed_at + a.nstage);
            for (int st = failed_at; st < issued_end; ++st)
                (void)mbar_wait_budget(&full[st % a.nstage], (unsigned)((st / a.nstage) & 1), budget);
        }
        return;
    }

    // add the ks lanes of each tile in a fixed order; lane 0 of the tile writes
    const G32Out& o = a.out[active ? a.to[tile] : 0];
    double* dst = part + chunk * a.part_stride + o.off;
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < TJ; ++v) {
            double r;
            if constexpr (DF) {
                r = (double)tot[u][v] + (double)cmp[u][v];
            } else {
                const float c = (v & 1) ? __high2float(cmpb[u][v / 2]) : __low2float(cmpb[u][v / 2]);
                r = (double)tot[u][v] - (double)c;
            }
            for (int off = a.ks >> 1; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
            const int i = i0 + u - o.lbase, j = j0 + v - o.rbase;
            if (active && kg == 0 && g32_need(o, i, j)) dst[i + (int64_t)o.ld * j] = r;
        }
}

// out(i, j) = sum over chunks of part[c * stride + off + i + ldp * j] in chunk order; one warp
// per entry.  sym: only i <= j is read and written to both (i, j) and (j, i).
__global__ void k_part_sum(int rows, int cols, int ldp, int64_t off, int64_t stride, int nparts,
                           const double* __restrict__ part, double* __restrict__ out, int ldo, int sym) {
    const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= (int64_t)rows * cols) return;
    const int i = (int)(e % rows), j = (int)(e / rows);
    if (sym && i > j) return;
    double s = 0.0;
    for (int c = lane; c < nparts; c += 32) s += part[c * stride + off + i + (int64_t)ldp * j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane) return;
    out[i + (int64_t)ldo * j] = s;
    if (sym) out[j + (int64_t)ldo * i] = s;
}

// G -= C^T C for the b x b matrix G and the w x b matrix C (column-major, ld ldc); one thread
// per entry.
__global__ void k_sub_ctc(int w, int b, const double* __restrict__ C, int ldc, double* __restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e % b, j = e / b;
    double s = 0.0;
    for (int k = 0; k < w; ++k) s = fma(C[k + (int64_t)ldc * i], C[k + (int64_t)ldc * j], s);
    G[i + (int64_t)b * j] -= s;
}

// K ((w + b) x b, column-major, ld w + b) = [-C Rinv; Rinv] for C (w x b, ld ldc) and the upper
// triangular Rinv (b x b, ld b): [L V] K = (V - L C) Rinv.  One thread per entry; skipped if
// *status & skip.
__global__ void k_projapply_coef(int w, int b, const double* __restrict__ C, int ldc, const double* __restrict__ Rinv,
                                 double* __restrict__ K, const unsigned* status, unsigned skip) {
    if (*status & skip) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = w + b;
    if (e >= q * b) return;
    const int i = e % q, c = e / q;
    double v = 0.0;
    if (i < w) {
        for (int k = 0; k <= c; ++k) v = fma(-C[i + (int64_t)ldc * k], Rinv[k + (int64_t)b * c], v);
    } else if (i - w <= c) {
        v = Rinv[(i - w) + (int64_t)b * c];
    }
    K[e] = v;
}

// ---------------------------------------------------------------- host side
// Tiles of TI x TJ staged columns covering every needed entry of the outputs.
void build_tiles(G32Args& a, int TI, int TJ) {
    a.ntiles = 0;
    for (int oi = 0; oi < a.nout; ++oi) {
        const G32Out& o = a.out[oi];
        for (int i0 = 0; i0 < o.rows; i0 += TI)
            for (int j0 = 0; j0 < o.cols; j0 += TJ) {
                bool need = false;
                for (int u = 0; u < TI && !need; ++u)
                    for (int v = 0; v < TJ && !need; ++v) need = g32_need(o, i0 + u, j0 + v);
                if (!need) continue;
                LG_REQUIRE(a.ntiles < kG32MaxTiles, LOBPCG_ERR_ARG, "Gram tile table overflow");
                a.ti[a.ntiles] = (uint16_t)(o.lbase + i0);
                a.tj[a.ntiles] = (uint16_t)(o.rbase + j0);
                a.to[a.ntiles] = (uint8_t)oi;
                ++a.ntiles;
            }
    }
}

template <bool DF>
void g32_launch(G32Args& a, int64_t n, int64_t ld, const G32Block* blk, int nblk, int Q, int nchunks,
                double* part, unsigned* status, cudaStream_t st) {
    constexpr int TI = TileShape<DF>::TI, TJ = TileShape<DF>::TJ;
    LG_REQUIRE(nblk <= kG32MaxBlocks, LOBPCG_ERR_ARG, "too many Gram blocks");
    a.nblk = 0;
    for (int b = 0; b < nblk; ++b) {
        if (blk[b].w <= 0) continue;
        LG_REQUIRE(blk[b].w <= 256, LOBPCG_ERR_ARG, "Gram block too wide");
        a.coff[a.nblk] = blk[b].coff;
        a.w[a.nblk] = blk[b].w;
        ++a.nblk;
    }
    a.Q = Q;
    a.K = (Q <= 128) ? 128 : 64;
    build_tiles(a, TI, TJ);
    if (a.ntiles == 0) return;
    // lanes per tile: more lanes when there are few tiles (at most 32, K >= 4 * ks)
    a.ks = 8;
    while (a.ks < 32 && a.ntiles * a.ks * 2 <= kG32Threads && 4 * a.ks * 2 <= a.K) a.ks *= 2;
    a.tpc = std::min(a.ntiles, kG32Threads / a.ks);
    a.ngroups = (a.ntiles + a.tpc - 1) / a.tpc;
    const int64_t stage_bytes = (int64_t)Q * a.K * sizeof(float);
    const int64_t budget = DF ? kG32SmemBudget : kG32SmemBudget / 2;    // two float32 blocks per SM
    a.nstage = (int)std::max<int64_t>(2, std::min<int64_t>(6, (budget - 2 * kG32Header) / stage_bytes));
    a.spin = stage_wait_polls();
    LG_REQUIRE(2 * kG32Header + a.nstage * stage_bytes <= 227 * 1024, LOBPCG_ERR_ARG, "Gram stage too large");
    a.rows_per_chunk = ceil_div(ceil_div(n, nchunks), 128) * 128;
    // encode the column blocks (rows beyond n read as zeros)
    int k = 0;
    for (int b = 0; b < nblk; ++b) {
        if (blk[b].w <= 0) continue;
        encode_f32_cols(&a.map[k++], blk[b].p, n, blk[b].w, ld, a.K);
    }
    const size_t smem = 2 * kG32Header + (size_t)a.nstage * stage_bytes;
    static std::atomic<unsigned long long> attr_set{0};   // one bit per device
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        LG_CUDA(cudaFuncSetAttribute(k_gram32<DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set.fetch_or(bit);
    }
    const int threads = (int)ceil_div((int64_t)a.tpc * a.ks, 32) * 32;
    k_gram32<DF><<<(unsigned)(nchunks * a.ngroups), threads, smem, st>>>(a, n, part, status);
    LG_CHECK_LAUNCH();
}

void part_sum(int rows, int cols, int ldp, int64_t off, int64_t stride, int nparts, const double* part,
              double* out, int ldo, bool sym, cudaStream_t st) {
    const int64_t threads = (int64_t)rows * cols * 32;
    k_part_sum<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(rows, cols, ldp, off, stride, nparts, part, out,
                                                                   ldo, sym ? 1 : 0);
    LG_CHECK_LAUNCH();
}

}  // namespace

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

void encode_f32_cols(CUtensorMap* map, const float* p, int64_t n, int w, int64_t ld, int box_rows, bool swizzle128) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    LG_REQUIRE(g_encode, LOBPCG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    LG_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0, LOBPCG_ERR_ARG,
               "float32 blocks must be 16-byte aligned with a leading dimension divisible by 4");
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)w};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)w};
    const cuuint32_t es[2] = {1, 1};
    LG_REQUIRE(!swizzle128 || box_rows * sizeof(float) == 128, LOBPCG_ERR_ARG, "128-byte swizzle needs 32-row boxes");
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), dims, strides, box,
                                es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LG_REQUIRE(r == CUDA_SUCCESS, LOBPCG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}


void encode_f64_cols(CUtensorMap* map, const double* p, int64_t n, int w, int64_t ld, int box_rows) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    LG_REQUIRE(g_encode, LOBPCG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    LG_REQUIRE((reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 2 == 0, LOBPCG_ERR_ARG,
               "float64 blocks must be 16-byte aligned with an even leading dimension");
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)w};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(double)};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)w};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(p), dims, strides, box,
                                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LG_REQUIRE(r == CUDA_SUCCESS, LOBPCG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

void launch_gram_sub_ctc(int w, int b, const double* C, int ldc, double* G, cudaStream_t st) {
    if (b <= 0 || w <= 0) return;
    k_sub_ctc<<<(unsigned)ceil_div((int64_t)b * b, 256), 256, 0, st>>>(w, b, C, ldc, G);
    LG_CHECK_LAUNCH();
}

void launch_projapply_coef(int w, int b, const double* C, int ldc, const double* Rinv, double* K,
                           const unsigned* status, unsigned skip, cudaStream_t st) {
    if (b <= 0) return;
    k_projapply_coef<<<(unsigned)ceil_div((int64_t)(w + b) * b, 128), 128, 0, st>>>(w, b, C, ldc, Rinv, K, status,
                                                                                   skip);
    LG_CHECK_LAUNCH();
}

int g32_chunks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 512), 2 * kNumSMs)); }

void launch_gram32_cross(int64_t n, int64_t ld, const float* S0, int w0, const float* S1, int w1, const float* V,
                         int b, double* C, double* G, double* part, int64_t part_doubles, unsigned* status,
                         int tc, cudaStream_t st) {
    const int wl = w0 + w1;
    if (b <= 0 || (wl == 0 && !G)) return;
    const int vb = ((wl + 7) / 8) * 8;
    const int Q = vb + ((b + 7) / 8) * 8;
    const G32Block blk[3] = {{S0, w0, 0}, {S1, w1, w0}, {V, b, vb}};
    static thread_local G32Args a;    // ~4 KB: keep it off the stack
    a = G32Args{};
    a.nout = 0;
    int64_t off = 0;
    if (wl > 0) {
        a.out[a.nout++] = G32Out{off, wl, 0, vb, wl, b, G32_ALL, 0, 0};
        off += (int64_t)wl * b;
    }
    int64_t goff = off;
    if (G) {
        a.out[a.nout++] = G32Out{off, b, vb, vb, b, b, G32_UPPER, 0, 0};
        off += (int64_t)b * b;
    }
    const int nchunks = g32_chunks(n);
    a.part_stride = off;
    LG_REQUIRE(nchunks * off <= part_doubles, LOBPCG_ERR_ARG, "Gram scratch too small");
    if (!launch_gram_tc(blk, 3, a.out, a.nout, off, n, ld, nchunks, part, status, tc, st))
        g32_launch<false>(a, n, ld, blk, 3, Q, nchunks, part, status, st);
    if (wl > 0) part_sum(wl, b, wl, 0, off, nchunks, part, C, wl, false, st);
    if (G) part_sum(b, b, b, goff, off, nchunks, part, G, b, true, st);
}

void launch_gram_mx2(int64_t n, int64_t ld, const float* Xh, const float* Xl, const float* W, const float* P,
                     const float* R, const float* AW, const float* AP, int m, int b, int bp, double* part,
                     int64_t part_doubles, const double* lam, double* gramA, double* gramB, unsigned* status,
                     int tc, cudaStream_t st) {
    const int q = m + b + bp;
    const int qp = ((q + 7) / 8) * 8;
    const int nchunks = g32_chunks(n);
    const int64_t q2 = (int64_t)q * q;
    LG_REQUIRE(nchunks * 2 * q2 <= part_doubles, LOBPCG_ERR_ARG, "Gram scratch too small");
    static thread_local G32Args a;
    // float32 tiles: S = [Xh W P] at 0, T = [R AW AP] at qp
    {
        a = G32Args{};
        const G32Block blk[6] = {{Xh, m, 0}, {W, b, m}, {P, bp, m + b}, {R, m, qp}, {AW, b, qp + m}, {AP, bp, qp + m + b}};
        a.nout = 2;
        a.out[0] = G32Out{0, q, 0, qp, q, q, G32_MXA, m, b};
        a.out[1] = G32Out{q2, q, 0, 0, q, q, G32_MXB, m, b};
        a.part_stride = 2 * q2;
        if (!launch_gram_tc(blk, 6, a.out, a.nout, a.part_stride, n, ld, nchunks, part, status, tc, st))
            g32_launch<false>(a, n, ld, blk, 6, 2 * qp, nchunks, part, status, st);
    }
    // double-float X^T X: hi plane at 0, lo plane at mp
    {
        a = G32Args{};
        const int mp = ((m + 7) / 8) * 8;
        const G32Block blk[2] = {{Xh, m, 0}, {Xl, m, mp}};
        a.nout = 1;
        a.out[0] = G32Out{q2, q, 0, 0, m, m, G32_UPPER, m, b};
        a.loff = mp;
        a.part_stride = 2 * q2;
        g32_launch<true>(a, n, ld, blk, 2, 2 * mp, nchunks, part, status, st);
    }
    launch_gram_finalize_mx(q, m, b, bp, nchunks, part, lam, gramA, gramB, st);
}

}  // namespace lg
