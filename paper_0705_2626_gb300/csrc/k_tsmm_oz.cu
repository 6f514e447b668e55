// Float64 products of a tall block and a small coefficient matrix, Y = S C, on the tensor cores
// by error-free digit products: the Ritz update of the Ritz update (Section 2.2) (X <- [X W P] C_X,
// P <- [W P] C_P, and the A-side) and the triangular applies V <- V R^-1 of the orthonormalisations of X and W and
// 14-15, in the float64 form.
//
// Each grid point p (a row of S, at most 32 columns; column k scaled by an exact power of two
// 2^a_k and row k of C by 2^-a_k, see TZ_SCALE_*) is written in the frame of its largest entry
// (|S(p, k)| < 2^E_p for every k) as
//     S(p, k) = 2^(E_p - 56) sum_{s=0..7} d_s(p, k) 2^(7 (7 - s)) + err,  |err| <= 2^(E_p - 57),
// with signed 7-bit digits d_s (oz_digits.cuh); each column j of C likewise in the frame of its
// largest entry F_j with digits e_t(k, j).  Digits are exact in bfloat16 and so are their
// products in float32.  With the level L = s + t,
//     Y(p, j) = 2^(E_p + F_j - 70) sum_{L=0..14} 2^(7 (8 - L)) D_L(p, j),
//     D_L(p, j) = sum_{s + t = L} sum_k d_s(p, k) e_t(k, j),
// and |D_L| <= 8 q 127^2 < 2^22 for q <= 32 columns, so every partial sum is an exact float32
// integer whatever the tensor cores' accumulator rounding.  One MMA forms all levels at once:
// the A operand holds the digit lines (K index 8 k + s) of 128 grid points, the B operand the
// Toeplitz expansion B(8 k + s, (L, j)) = e_{L-s}(k, j) of C, so that TMEM lane p, column
// (L, j) receives D_L(p, j).  Levels L <= 8 are kept (the rest lie below 2^-55 of
// max_k |S(p, k)| max_k |C(k, j)|); each output is assembled from its nine levels in 64-bit
// integers and rounded to float64 once.  This is Ozaki, Ogita and Oishi's error-free splitting
// ("Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012) with a common exponent per
// row of S and per column of C, and the digit levels of one output summed by the MMA itself.
//
// Warp roles (18 warps, one block per SM, persistent over 128-point tiles): warps 0-7 split,
// as two groups of 4 warps that take alternate tiles (thread = grid point, all columns of its
// row); warps 8-15 drain the accumulators, as two groups that take alternate tiles and
// accumulator buffers (TMEM lane quarter warp % 4, thread = grid point, all outputs of its row);
// warp 16 streams the float64 tiles in with TMA; warp 17 owns the tensor memory and issues the
// MMAs.  The two accumulator buffers let the drain of one tile overlap the MMAs of the next.  Every
// tile of S is read in full before any output of that tile is written, so Y may overwrite S in
// place (thread blocks own disjoint tiles).  Every wait is bounded (status bit ST_TIMEOUT).
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "oz_digits.cuh"
#include "tma.cuh"

namespace lg {
namespace {

constexpr int kTzTile = 128;                   // grid points per tile (MMA M, TMEM lanes)
constexpr int kTzLevels = 9;                   // digit levels kept, L = 0..8
constexpr int kTzMaxQ = 32;                    // columns of S (exact level sums need q <= 32)
constexpr int kTzMaxOut = 28;                  // outputs: 9 x (outputs rounded up to 4) <= 256
constexpr int kTzSplitWarps = 8;
constexpr int kTzEpiWarps = 8;
constexpr int kTzTmaWarp = kTzSplitWarps + kTzEpiWarps;
constexpr int kTzMmaWarp = kTzTmaWarp + 1;
constexpr int kTzThreads = 32 * (kTzMmaWarp + 1);
constexpr int kTzEpRing = 4;                   // row-exponent slots (tiles in flight)
constexpr int kTzSmemMax = 227 * 1024;
constexpr int kTzNaN = 1 << 29;                // row / column frame of a non-finite entry
constexpr int kTzOff = 1 << 20;                // scale of a column that meets only zero coefficients

struct TzArgs {
    CUtensorMap map[3];          // float64 column blocks of S, boxes of 128 points x w columns
    int coff[3];                 // first column of each block
    int nblk;
    int q, q2;                   // columns of S; rounded up to even (MMA K steps of 2 columns)
    int nka;                     // 128-byte K atoms (8 columns of digit lines each)
    int nx, np, w0p;             // outputs: nx from all rows of C, then np from rows >= w0p
    int nout, nj, N;             // nx + np; rounded up to 4; MMA N = 9 nj rounded up to 16
    int ldc;
    const double* C;             // q x nx coefficients, column-major, leading dimension ldc
    double* out0;                // the nx outputs, leading dimension ldout
    double* out1;                // the np outputs
    int64_t ldout, n, ntiles;
    int nf, na;                  // float64 staging slots, digit stages
    int tmem_cols;
    int polls;
    unsigned skip;
    int scale_mode;              // TZ_SCALE_*
    const int* sexp;             // TZ_SCALE_S_COLS: largest exponent field of each column of S
    int b_bytes, a_bytes, f_bytes;
};

__device__ __forceinline__ void tz_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tz_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tz_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tz_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait that gives up early once another role has flagged a failure.
__device__ __forceinline__ bool tz_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag, int polls) {
#pragma unroll 1
    for (int it = 0; it < polls; ++it) {
        if (mbar_poll(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled layout, 8-line groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (bits 46-48), swizzle mode 2
// (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t tz_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tz_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tz_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tz_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 lanes x 4 consecutive 32-bit columns (the caller waits once for several loads).
__device__ __forceinline__ void tz_ld4(uint32_t taddr, float (&r)[4]) {
    uint32_t u0, u1, u2, u3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(u0), "=r"(u1), "=r"(u2), "=r"(u3)
                 : "r"(taddr)
                 : "memory");
    r[0] = __uint_as_float(u0);
    r[1] = __uint_as_float(u1);
    r[2] = __uint_as_float(u2);
    r[3] = __uint_as_float(u3);
}
__device__ __forceinline__ void tz_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 lanes x 8 consecutive 32-bit columns.
__device__ __forceinline__ void tz_ld8(uint32_t taddr, float (&r)[8]) {
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}

// Biased exponent field of x (0 for zeros and subnormals, 2047 for infinities and NaNs).
__device__ __forceinline__ int exp_field(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// The 8 digits of x in the frame of the exponent field emax >= exp_field(x) (oz_digits) as
// bfloat16, digit s in the (s & 1) half of word s / 2: one 16-byte chunk of digit lines.
__device__ __forceinline__ uint4 digits8(double x, int emax) {
    float d[8];
    oz_digits(x, emax, d);
    return make_uint4(oz_pack2(d[0], d[1]), oz_pack2(d[2], d[3]), oz_pack2(d[4], d[5]), oz_pack2(d[6], d[7]));
}

// t 2^ex rounded to float64 (nearest, ties to even): the conversion of t is the one rounding
// (on the otherwise idle float64 pipe), the power of two is added to the exponent field; results
// below the normal range are flushed to zero, results above it become infinities.
__device__ __forceinline__ double scaled_to_double(long long t, int ex) {
    const double y = __ll2double_rn(t);
    const int hi = __double2hiint(y), lo = __double2loint(y);
    const int e = ((hi >> 20) & 0x7FF) + ex;           // biased exponent of the result
    const int sgn = hi & (int)0x80000000u;
    const bool over = e >= 2047, under = e <= 0 || t == 0;
    int rh = hi + (int)((unsigned)ex << 20);
    rh = over ? (sgn | 0x7FF00000) : rh;
    rh = under ? sgn : rh;
    return __hiloint2double(rh, (over || under) ? 0 : lo);
}

// One output from its nine levels D_0..D_8 (exact float32 integers, |D| < 2^22):
// T = sum_L D_L 2^(7 (8 - L)), result = round(T / 2^14) 2^(E_p + F_j - 56) rounded to float64
// (the 14 bits rounded off lie 2^-57 below max |S(p, .)| max |C(., j)|; rounding to nearest
// rather than down keeps the outputs free of a common bias).  ex = E_p + F_j - 56.
__device__ __forceinline__ double combine_levels(const float (&D)[kTzLevels], int ex) {
    // b_L = bits of D_L + 1.5 2^23 = 0x4B400000 + D_L exactly (|D_L| < 2^22); the bias is taken
    // out of each combination at once (32-bit wrap-around: every combination fits in 32 bits)
    constexpr unsigned kB = 0x4B400000u;
    unsigned b[kTzLevels];
#pragma unroll
    for (int L = 0; L < kTzLevels; ++L) b[L] = __float_as_uint(D[L] + 12582912.0f);
    const int lo14 = (int)(b[5] * 128u + b[6] - 129u * kB) +
                     ((int)(b[7] * 128u + b[8] + (8192u - 129u * kB)) >> 14);   // floor(x + 1/2)
    const int a1 = (int)(b[0] * 128u + b[1] - 129u * kB);
    const int a2 = (int)(b[2] * 128u + b[3] - 129u * kB);
    const int i4 = (int)(b[4] - kB);
    const long long t = (long long)a1 * (1ll << 35) + (long long)a2 * (1ll << 21) + (long long)i4 * (1ll << 14) +
                        (long long)lo14;
    return scaled_to_double(t, ex);
}

// Entry (k, j) of the coefficient matrix as the kernel applies it.
__device__ __forceinline__ double coef(const TzArgs& a, int k, int j) {
    if (k >= a.q) return 0.0;
    if (j < a.nx) return a.C[k + (int64_t)a.ldc * j];
    return k >= a.w0p ? a.C[k + (int64_t)a.ldc * (j - a.nx)] : 0.0;
}

// Byte offset of the 16-byte chunk (line r, column k) of a K-major operand in the 128-byte
// swizzled layout with `lines` lines per K atom of 8 columns.
__device__ __forceinline__ uint32_t chunk_off(int r, int k, int lines) {
    return (uint32_t)((k >> 3) * lines * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((((k & 7) ^ (r & 7))) << 4));
}

// Tiles are processed in order t = 0, 1, ... (tile blockIdx.x + t gridDim.x); split group g and
// drain group g (4 warps each, thread = grid point) take the tiles t = g mod 2, the drain group
// reading accumulator buffer g.  Every staging slot, digit stage and exponent slot is used by one
// group only (even ring sizes), so no parity wait runs two phases ahead of its barrier.
__global__ void __launch_bounds__(kTzThreads, 1) k_tsmm_oz(const __grid_constant__ TzArgs a, unsigned* status) {
    extern __shared__ unsigned char tz_smem_raw[];
    unsigned char* smem = tz_smem_raw + ((1024 - (smem_addr(tz_smem_raw) & 1023)) & 1023);
    unsigned char* sB = smem;
    unsigned char* sA = smem + a.b_bytes;
    double* sF = reinterpret_cast<double*>(sA + (size_t)a.na * a.a_bytes);
    const int f_doubles = a.f_bytes / 8;
    int* ep = reinterpret_cast<int*>(sF + (size_t)a.nf * f_doubles);      // [kTzEpRing][kTzTile]
    int* colexp = ep + kTzEpRing * kTzTile;                                  // [32] frame of each output
    int* aoff = colexp + 32;                                                 // [32] scale exponent a_k
    uint64_t* sfull = reinterpret_cast<uint64_t*>(colexp + 64);
    uint64_t* sempty = sfull + 4;
    uint64_t* afull = sempty + 4;
    uint64_t* aempty = afull + 2;
    uint64_t* accfull = aempty + 2;
    uint64_t* accempty = accfull + 2;
    uint64_t* epfull = accempty + 2;
    uint64_t* fin = epfull + kTzEpRing;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    int* skip_flag = reinterpret_cast<int*>(tslot + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = (int)((a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    if (tid == 0) {
        for (int i = 0; i < a.nf; ++i) {
            mbar_init(&sfull[i], 1);
            mbar_init(&sempty[i], 4);
        }
        for (int i = 0; i < a.na; ++i) {
            mbar_init(&afull[i], 4);
            mbar_init(&aempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accfull[i], 1);
            mbar_init(&accempty[i], 4);
        }
        for (int i = 0; i < kTzEpRing; ++i) mbar_init(&epfull[i], 4);
        mbar_init(fin, 1);
        *abort_flag = 0;
        *skip_flag = (status && (*status & a.skip)) ? 1 : 0;
        mbar_fence_init();
    }
    // column scales 2^a_k: S(:, k) 2^a_k, C(k, :) 2^-a_k
    if (tid < a.q) {
        int ak = 0;
        if (a.scale_mode == TZ_SCALE_C_ROWS) {
            int em = 0;
            for (int j = 0; j < a.nout; ++j) em = max(em, exp_field(coef(a, tid, j)));
            ak = em == 0 ? -kTzOff : em - 1023;          // a zero row: the column takes no part
        } else if (a.scale_mode == TZ_SCALE_S_COLS) {
            const int es = a.sexp[tid];
            ak = (es == 0 || es == 2047) ? 0 : 1023 - es;
        }
        aoff[tid] = ak;
    }
    __syncthreads();
    // frame of every output column: the largest scaled exponent field of its coefficients
    if (tid < a.nout) {
        int em = -kTzOff;
        bool bad = false;
        for (int k = 0; k < a.q; ++k) {
            const int e = exp_field(coef(a, k, tid));
            bad |= e == 2047;
            if (e != 0) em = max(em, e - aoff[k]);
        }
        colexp[tid] = bad ? kTzNaN : em;
    }
    __syncthreads();
    if (*skip_flag) return;
    if (warp == kTzMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // B operand: the Toeplitz expansion of the coefficient digits, line (L, j) = L nj + j
    for (int idx = tid; idx < a.N * a.q2; idx += kTzThreads) {
        const int nl = idx / a.q2, k = idx - nl * a.q2;
        const int L = nl / a.nj, j = nl - L * a.nj;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (L < kTzLevels && j < a.nout && k < a.q && colexp[j] != kTzNaN) {
            const uint4 d = digits8(coef(a, k, j), colexp[j] + aoff[k]);
            const uint32_t dw[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const int t = L - s;
                const uint32_t v = (t >= 0 && t < 8) ? ((dw[t >> 1] >> (16 * (t & 1))) & 0xFFFFu) : 0u;
                w[s >> 1] |= v << (16 * (s & 1));
            }
        }
        *reinterpret_cast<uint4*>(sB + chunk_off(nl, k, a.N)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    tz_fence_proxy_async();
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    const uint32_t tmem = *tslot;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
    };

    if (warp < kTzSplitWarps) {
        // ------------------------------------------------------------------ split
        const int g = warp >> 2, p = 32 * (warp & 3) + lane;
        bool ok = true;
        for (int t = g; t < nt; t += 2) {
            const int fs = t % a.nf, as = t % a.na;
            // the staged tile, and the digit stage (and, through the MMAs of tile t - 2, the drain
            // of tile t - 4, which read this tile's exponent slot)
            if (!__all_sync(0xffffffffu, tz_wait(&sfull[fs], (unsigned)((t / a.nf) & 1), abort_flag, a.polls)) ||
                (t >= a.na &&
                 !__all_sync(0xffffffffu,
                             tz_wait(&aempty[as], (unsigned)(((t / a.na) - 1) & 1), abort_flag, a.polls)))) {
                ok = false;
                break;
            }
            const double* stg = sF + (size_t)fs * f_doubles + p;
            // frame of the grid point: its largest scaled exponent field (zeros take no part)
            int em = -kTzOff, eraw = 0;
#pragma unroll 8
            for (int k = 0; k < a.q; ++k) {
                const int e = (reinterpret_cast<const int*>(stg + k * kTzTile)[1] >> 20) & 0x7FF;
                eraw = max(eraw, e);
                em = max(em, e != 0 ? e + aoff[k] : -kTzOff);
            }
            ep[(t % kTzEpRing) * kTzTile + p] = eraw == 2047 ? kTzNaN : em;
            unsigned char* stA = sA + (size_t)as * a.a_bytes;
#pragma unroll 8
            for (int k = 0; k < a.q2; ++k) {
                const double x = k < a.q ? stg[k * kTzTile] : 0.0;
                *reinterpret_cast<uint4*>(stA + chunk_off(p, k, kTzTile)) = digits8(x, k < a.q ? em - aoff[k] : 0);
            }
            tz_fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                tz_arrive(&sempty[fs]);
                tz_arrive(&epfull[t % kTzEpRing]);
                tz_arrive(&afull[as]);
            }
        }
        if (!ok && lane == 0) fail();
    } else if (warp < kTzTmaWarp) {
        // ------------------------------------------------------------------ drain
        const int g = (warp - kTzSplitWarps) >> 2, quarter = warp & 3, p = 32 * quarter + lane;
        const uint32_t tbase = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(g * a.N);
        bool ok = true;
        for (int t = g; t < nt; t += 2) {
            if (!__all_sync(0xffffffffu, tz_wait(&accfull[g], (unsigned)((t >> 1) & 1), abort_flag, a.polls)) ||
                !__all_sync(0xffffffffu,
                            tz_wait(&epfull[t % kTzEpRing], (unsigned)((t / kTzEpRing) & 1), abort_flag, a.polls))) {
                ok = false;
                break;
            }
            tz_fence_after();
            const int em = ep[(t % kTzEpRing) * kTzTile + p];
            const int64_t P = ((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * kTzTile + p;
            const bool valid = P < a.n;
            // outputs c .. c + W - 1 from their nine levels
            auto drain = [&](int c, auto width) {
                constexpr int W = decltype(width)::value;
                float v[kTzLevels][W];
#pragma unroll
                for (int L = 0; L < kTzLevels; ++L) {
                    if constexpr (W == 8) tz_ld8(tbase + (uint32_t)(L * a.nj + c), v[L]);
                    else tz_ld4(tbase + (uint32_t)(L * a.nj + c), v[L]);
                }
                tz_wait_ld();
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int j = c + u;
                    if (j >= a.nout || !valid) continue;
                    float D[kTzLevels];
#pragma unroll
                    for (int L = 0; L < kTzLevels; ++L) D[L] = v[L][u];
                    const int cj = colexp[j];
                    const double y = (em == kTzNaN || cj == kTzNaN) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                     : combine_levels(D, em + cj - 2100);
                    double* dst = j < a.nx ? a.out0 + (int64_t)j * a.ldout : a.out1 + (int64_t)(j - a.nx) * a.ldout;
                    dst[P] = y;
                }
            };
            int c = 0;
            if ((a.nj & 7) == 0) {         // 8-column loads stay 8-aligned in every level
#pragma unroll 1
                for (; c < a.nj; c += 8) drain(c, std::integral_constant<int, 8>());
            }
#pragma unroll 1
            for (; c < a.nj; c += 4) drain(c, std::integral_constant<int, 4>());
            tz_fence_before();
            __syncwarp();
            if (lane == 0) tz_arrive(&accempty[g]);
        }
        if (!ok && lane == 0) fail();
    } else if (warp == kTzTmaWarp) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < nt; ++t) {
                const int fs = t % a.nf;
                if (t >= a.nf && !tz_wait(&sempty[fs], (unsigned)(((t / a.nf) - 1) & 1), abort_flag, a.polls)) {
                    fail();
                    break;
                }
                const int x = (int)(((int64_t)blockIdx.x + (int64_t)t * gridDim.x) * kTzTile);
                mbar_expect_tx(&sfull[fs], (unsigned)(a.q * kTzTile * 8));
                double* dst = sF + (size_t)fs * f_doubles;
                for (int b = 0; b < a.nblk; ++b) tma_load_2d(dst + a.coff[b] * kTzTile, &a.map[b], x, 0, &sfull[fs]);
                issued = t + 1;
            }
            // the copies still in flight land before the block exits
            int budget = kSpinLimit;
            for (int t = std::max(0, issued - a.nf); t < issued; ++t)
                if (!mbar_wait_budget(&sfull[t % a.nf], (unsigned)((t / a.nf) & 1), budget)) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
        }
    } else {
        // ------------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = tz_idesc(kTzTile, a.N);
            const uint32_t bA = smem_addr(sA), bB = smem_addr(sB);
            const int nk = a.q2 / 2;
            for (int t = 0; t < nt; ++t) {
                const int as = t % a.na, buf = t & 1;
                if (!tz_wait(&afull[as], (unsigned)((t / a.na) & 1), abort_flag, a.polls) ||
                    (t >= 2 && !tz_wait(&accempty[buf], (unsigned)(((t >> 1) - 1) & 1), abort_flag, a.polls))) {
                    fail();
                    break;
                }
                tz_fence_after();
                const uint32_t sa = bA + (uint32_t)(as * a.a_bytes);
#pragma unroll 1
                for (int kk = 0; kk < nk; ++kk) {
                    const uint32_t ka = (uint32_t)((kk >> 2) * (kTzTile * 128) + (kk & 3) * 32);
                    const uint32_t kb = (uint32_t)((kk >> 2) * (a.N * 128) + (kk & 3) * 32);
                    tz_mma(tmem + (uint32_t)(buf * a.N), tz_desc(sa + ka), tz_desc(bB + kb), idesc, kk > 0 ? 1u : 0u);
                }
                tz_commit(&aempty[as]);
                tz_commit(&accfull[buf]);
            }
            // every MMA issued so far has completed once `fin` flips (this wait ignores the abort
            // flag: the tensor memory is released only after them)
            tz_commit(fin);
            if (!mbar_wait(fin, 0u)) atomicOr(status, ST_TIMEOUT | ST_TIMEOUT_MMA);
        }
    }
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    if (warp == kTzMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

}  // namespace

bool tsmm_oz_fits(int q, int nout) { return q >= 1 && q <= kTzMaxQ && nout >= 1 && nout <= kTzMaxOut; }

bool launch_tsmm_oz(int64_t n, const Blocks3& S, const double* C, int ldc, int nx, int np, int w0p, double* out0,
                    double* out1, int64_t ldout, unsigned* status, unsigned skip, cudaStream_t st, int scale_mode,
                    const int* sexp) {
    const int q = S.q();
    if (!tsmm_oz_fits(q, nx + np) || n < kTzTile || S.ld % 2 != 0 || !status) return false;
    if (S.t0 != DT_F64 || (S.w[1] + S.w[2] > 0 && S.t12 != DT_F64)) return false;
    for (int b = 0; b < 3; ++b)
        if (S.w[b] > 0 && (reinterpret_cast<uintptr_t>(S.p[b]) & 15) != 0) return false;
    static thread_local TzArgs a;
    a = TzArgs{};
    a.q = q;
    a.q2 = q + (q & 1);
    a.nka = (a.q2 + 7) / 8;
    a.nx = nx;
    a.np = np;
    a.w0p = w0p;
    a.nout = nx + np;
    a.nj = (a.nout + 3) / 4 * 4;
    a.N = (kTzLevels * a.nj + 15) / 16 * 16;
    a.ldc = ldc;
    a.C = C;
    a.out0 = out0;
    a.out1 = out1 ? out1 : out0;
    a.ldout = ldout;
    a.n = n;
    a.ntiles = ceil_div(n, (int64_t)kTzTile);
    a.skip = skip;
    a.scale_mode = (scale_mode == TZ_SCALE_S_COLS && !sexp) ? TZ_SCALE_NONE : scale_mode;
    a.sexp = sexp;
    a.polls = stage_wait_polls();
    a.b_bytes = a.nka * a.N * 128;
    a.a_bytes = a.nka * kTzTile * 128;
    a.f_bytes = q * kTzTile * 8;
    const int misc = kTzEpRing * kTzTile * 4 + 64 * 4 + 32 * 8 + 64;
    // two digit stages and 2 or 4 staging slots (even rings: every slot belongs to one group)
    a.na = 2;
    int best = 0;
    for (int nf = 4; nf >= 2 && !best; nf -= 2) {
        const int total = 1024 + a.b_bytes + a.na * a.a_bytes + nf * a.f_bytes + misc;
        if (total <= kTzSmemMax) {
            a.nf = nf;
            best = total;
        }
    }
    if (!best) return false;
    int cols = 32;
    while (cols < 2 * a.N) cols *= 2;
    a.tmem_cols = cols;
    int k = 0, c = 0;
    for (int b = 0; b < 3; ++b) {
        if (S.w[b] > 0) {
            encode_f64_cols(&a.map[k], static_cast<const double*>(S.p[b]), n, S.w[b], S.ld, kTzTile);
            a.coff[k] = c;
            ++k;
        }
        c += S.w[b];
    }
    a.nblk = k;
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        LG_CUDA(cudaFuncSetAttribute(k_tsmm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kTzSmemMax));
        attr_set.fetch_or(bit);
    }
    const int64_t grid = std::min<int64_t>(a.ntiles, (int64_t)kNumSMs);
    k_tsmm_oz<<<(unsigned)grid, kTzThreads, (size_t)best, st>>>(a, status);
    LG_CHECK_LAUNCH();
    return true;
}

}  // namespace lg
