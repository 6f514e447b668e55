// Float64 Gram matrices of the Rayleigh-Ritz basis on the tensor cores (Section 2.2, the float64
// form) by error-free digit products.
//
// GB300 runs float64 fused multiply-adds at 2 per clock per SM; its bfloat16 tensor cores are
// about three orders of magnitude faster.  Within a window of kOzWindow grid points every
// float64 column c is written as
//     x = 2^(E_c - 56) sum_{s=0..7} d_s 2^(7 (7 - s)) + err,   |err| <= 2^(E_c - 57),
// with E_c fixed by the largest exponent of the column in the window (|x| < 2^E_c) and integer
// digits d_s = sign(x) * (bits 49 - 7 s .. 55 - 7 s of the 56-bit magnitude |x| 2^(56 - E_c),
// rounded to an integer), |d_s| <= 127.
// A digit is exact in bfloat16, a product of two digits (< 2^14) is exact in float32, and so
// is every partial sum of up to 1024 of them (< 2^24): the tensor cores, whatever their
// rounding of the float32 accumulator, then form every digit-pair sum
//     D_st(i, j) = sum_p d_s(x_i(p)) d_t(y_j(p))
// exactly, one TMEM accumulator per pair, over a window of 1024 points.  The window's share of
// the entry,
//     sum_p x_i y_j = 2^(E_i + E_j - 112) sum_{s,t} D_st 2^(7 (14 - s - t)),
// is formed in 64-bit integer arithmetic (truncated at 2^-62 of its largest possible value); the
// shares of the 16 windows of one exponent window are summed exactly in 128-bit integers and
// added, converted to float64 once, to the entry's float64 total.  This is the splitting method
// of Ozaki, Ogita and Oishi ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012) with a
// common exponent per column and window and every digit pair kept: the per-window result carries
// about 2^-56 of the window's largest products, below the rounding of a float64 dot product.
//
// Operands (the K dimension is the grid point): A = the digit lines of the left block L = S, line
// 8 i + s = digit s of column i (M = 128 lines per tile, up to 3 tiles); B = the digit lines of a
// group J of columns of the right block R = [S AS] (or S), line 8 j + t.  D(8 i + s, 8 j + t) =
// D_st(i, j).  Both operands sit in shared memory in the 128-byte swizzled K-major layout (one
// 128-byte line = 64 points of one digit line), written by the split warps.
//
// The largest exponent of every column over each exponent window of kOzExpPts points (16
// accumulation windows) comes from a first pass, k_oz_exponents, which reads the blocks once.
//
// Warp roles (21 warps, one block per SM): warps 0-15 split a stage of 64 points of their
// columns into digit lines (each lane copies its two points of the stages ahead into a ring in
// shared memory with cp.async, so the global-memory latency stays hidden), warps 16-19 drain the
// accumulators at the end of each window (TMEM lane quarters 0-3), warp 20 allocates the tensor
// memory and one of its threads issues the MMAs.  The thread blocks (chunk, g) of one row range
// share the left block and take different groups J of right columns, balanced between S and AS
// columns; they write their per-chunk partial sums in the layout of the float64 SIMT Gram, so the
// same fixed-order chunk sums finish the job.  Every wait is bounded (status bit ST_TIMEOUT).
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "oz_digits.cuh"
#include "tma.cuh"

namespace lg {
namespace {

constexpr int kOzDigits = 8;
constexpr int kOzStagePts = 64;                  // one 128-byte line of bfloat16 per digit line
constexpr int kOzWindowStages = 16;              // 1024 points per exact accumulation window
constexpr int kOzSplitWarps = 16;
constexpr int kOzEpiWarps = 4;
constexpr int kOzThreads = 32 * (kOzSplitWarps + kOzEpiWarps + 1);
constexpr int kOzMmaWarp = kOzSplitWarps + kOzEpiWarps;
constexpr int kOzMaxQ = 48;                      // left columns (3 A tiles of 16 columns)
constexpr int kOzMaxJ = 32;                      // right columns per thread block (N <= 256)
constexpr int kOzMaxGroups = 16;
constexpr int kOzMaxSplitCols = kOzMaxQ + kOzMaxJ;
constexpr int kOzColsPerWarp = (kOzMaxSplitCols + kOzSplitWarps - 1) / kOzSplitWarps;
constexpr int kOzExpPts = 16384;                 // points per exponent window
constexpr int kOzSmemBudget = 218 * 1024;

struct OzArgs {
    const double* R[2 * kOzMaxQ];    // right columns R = [S AS] (or S); the left block L = S = R[0, q)
    const int* ex;                   // largest exponent field of R column c over exponent window w: ex[w r + c]
    int q, r;                        // left / right column counts
    int nmt;                         // A tiles of 128 digit lines
    int ngroups;
    int jn[kOzMaxGroups];            // right columns of group g ...
    int16_t jidx[kOzMaxGroups][kOzMaxJ];   // ... R column of its B lines 8 j .. 8 j + 7
    int nb;                          // B lines (8 max jn rounded up to 32)
    int nstage;                      // digit stages in the ring
    int cpw;                         // split columns per warp (largest over the groups)
    int tmem_cols;
    int64_t n, rows_per_chunk, part_stride;
};

// Largest exponent field of each R column over each exponent window: one warp per (window,
// column), the high words of the column's values.  colmax (may be null): the largest over all
// windows, per column (zeroed by the caller).
__global__ void __launch_bounds__(256) k_oz_exponents(const __grid_constant__ OzArgs a, int* __restrict__ ex,
                                                      int* __restrict__ colmax) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.y * 8 + warp;
    if (c >= a.r) return;
    const int64_t p0 = (int64_t)blockIdx.x * kOzExpPts;
    const int64_t p1 = min(a.n, p0 + kOzExpPts);
    const int* src = reinterpret_cast<const int*>(a.R[c]);
    int mx = 0;
    for (int64_t base = p0; base < p1; base += 32 * 16) {
        int hw[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int64_t p = base + lane + 32 * k;
            hw[k] = p < p1 ? __ldg(src + 2 * p + 1) : 0;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) mx = max(mx, (hw[k] >> 20) & 0x7FF);
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        ex[(int64_t)blockIdx.x * a.r + c] = mx;
        if (colmax) atomicMax(colmax + c, mx);
    }
}

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---- tcgen05 / mbarrier helpers ----------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait that gives up early once another role has flagged a failure.  sleep_ns > 0: the
// waiting warp naps between polls (roles that wait long, so that they leave the issue slots to the
// split warps).
__device__ __forceinline__ bool oz_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                        unsigned sleep_ns = 0) {
#pragma unroll 1
    for (int it = 0; it < kSpinLimit; ++it) {
        if (mbar_poll(bar, parity)) return true;
        if (*abort_flag) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return false;
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled layout, 8-line groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (bits 46-48), swizzle mode 2
// (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns (no wait: the caller waits once for several loads).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// NF: float64 stages in the copy ring (NF - 1 stages of copies in flight ahead of the split).
template <int NF>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_gram_oz(const __grid_constant__ OzArgs a, double* __restrict__ part, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    const int g = blockIdx.y;
    const int jn = a.jn[g];
    const int a_bytes = a.nmt * 128 * 128;             // A tiles of one stage
    const int stage_bytes = a_bytes + a.nb * 128;
    const int fwarp_doubles = a.cpw * kOzStagePts;     // one split warp's float64 stage
    double* fring = reinterpret_cast<double*>(smem + (size_t)a.nstage * stage_bytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(fring + (size_t)NF * kOzSplitWarps * fwarp_doubles);
    uint64_t* empty = full + a.nstage;
    uint64_t* accfull = empty + a.nstage;
    uint64_t* accempty = accfull + 1;
    uint64_t* fin = accempty + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    int* nsplit_s = reinterpret_cast<int*>(tslot + 2);
    int16_t* srcidx = reinterpret_cast<int16_t*>(tslot + 4);   // split column -> R column
    int16_t* bline = srcidx + kOzMaxSplitCols;                 // split column -> B line group or -1

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = blockIdx.x * a.rows_per_chunk;
    const int64_t r1 = min(a.n, r0 + a.rows_per_chunk);
    const int64_t npts = r1 > r0 ? r1 - r0 : 0;
    const int nst = (int)((npts + kOzStagePts - 1) / kOzStagePts);
    const int nwin = (nst + kOzWindowStages - 1) / kOzWindowStages;

    if (tid == 0) {
        // split columns: the left columns 0..q-1 (their A lines; the B lines too when the column
        // is in J), then the AS columns of J
        int ns = a.q;
        for (int c = 0; c < a.q; ++c) {
            srcidx[c] = (int16_t)c;
            bline[c] = -1;
        }
        for (int j = 0; j < jn; ++j) {
            const int jr = a.jidx[g][j];
            if (jr < a.q) {
                bline[jr] = (int16_t)j;
            } else {
                srcidx[ns] = (int16_t)jr;
                bline[ns] = (int16_t)j;
                ++ns;
            }
        }
        *nsplit_s = ns;
        // split warps without a column take no part (a stage is full once the others arrive)
        for (int st = 0; st < a.nstage; ++st) {
            mbar_init(&full[st], (unsigned)min(kOzSplitWarps, ns));
            mbar_init(&empty[st], 1);
        }
        mbar_init(accfull, 1);
        mbar_init(accempty, kOzEpiWarps);
        mbar_init(fin, 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == kOzMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nsplit = *nsplit_s;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
    };

    if (warp < kOzSplitWarps && warp < nsplit) {
        // ------------------------------------------------------------------ split warps
        // Byte offsets, inside an 8-line group, of this lane's two points of digit line s
        // (128-byte swizzle: 16-byte chunk c of line s at chunk c ^ s).
        uint32_t soff[kOzDigits];
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s)
            soff[s] = (uint32_t)(s * 128 + ((((lane >> 2) ^ s) << 4) | ((4 * lane) & 15)));
        double* myring = fring + (size_t)warp * fwarp_doubles + 2 * lane;
        const size_t fstride = (size_t)kOzSplitWarps * fwarp_doubles;   // one float64 stage
        // this warp's columns, held in registers: the column, the byte offsets of its A and B
        // lines in a stage (-1: none), its R index
        const int ncw = min(a.cpw, (nsplit - warp + kOzSplitWarps - 1) / kOzSplitWarps);
        const double* csrc[kOzColsPerWarp];
        int coffa[kOzColsPerWarp], coffb[kOzColsPerWarp], cidx[kOzColsPerWarp];
#pragma unroll
        for (int u = 0; u < kOzColsPerWarp; ++u) {
            const int c = warp + u * kOzSplitWarps;
            const bool has = u < ncw;
            cidx[u] = has ? srcidx[c] : 0;
            csrc[u] = a.R[cidx[u]];
            coffa[u] = (has && c < a.q) ? (c >> 4) * 16384 + (c & 15) * 1024 : -1;
            coffb[u] = (has && bline[c] >= 0) ? a_bytes + bline[c] * 1024 : -1;
        }
        // copies of stage tt into float64 slot tt % NF: this lane's two points per column
        auto issue = [&](int tt) {
            if (tt < nst) {
                double* dst = myring + (size_t)(tt % NF) * fstride;
                const int64_t p0 = r0 + (int64_t)tt * kOzStagePts + 2 * lane;
#pragma unroll
                for (int u = 0; u < kOzColsPerWarp; ++u) {
                    if (u >= ncw) break;
                    if (p0 < r1) cp_async8(dst + u * kOzStagePts, csrc[u] + p0);
                    if (p0 + 1 < r1) cp_async8(dst + u * kOzStagePts + 1, csrc[u] + p0 + 1);
                }
            }
            cp_async_commit();
        };
        for (int tt = 0; tt < NF - 1; ++tt) issue(tt);
        int e[kOzColsPerWarp];
        int64_t ew_cur = -1;
        bool ok = true;
        for (int t = 0; t < nst && ok; ++t) {
            issue(t + NF - 1);
            cp_async_wait<NF - 1>();                 // the copies of stage t have landed
            const int slot = t % a.nstage;
            const int64_t p0 = r0 + (int64_t)t * kOzStagePts + 2 * lane;
            const int64_t ew = (r0 + (int64_t)t * kOzStagePts) / kOzExpPts;
            if (ew != ew_cur) {
                ew_cur = ew;
#pragma unroll
                for (int u = 0; u < kOzColsPerWarp; ++u) e[u] = u < ncw ? __ldg(a.ex + ew * a.r + cidx[u]) : 0;
            }
            if (t >= a.nstage &&
                !__all_sync(0xffffffffu, oz_wait(&empty[slot], (unsigned)((t / a.nstage - 1) & 1), abort_flag, 64))) {
                ok = false;
                break;
            }
            unsigned char* sst = smem + (size_t)slot * stage_bytes;
            const double* fsrc = myring + (size_t)(t % NF) * fstride;
#pragma unroll
            for (int u = 0; u < kOzColsPerWarp; ++u) {
                if (u >= ncw) break;
                const double x0 = p0 < r1 ? fsrc[u * kOzStagePts] : 0.0;
                const double x1 = p0 + 1 < r1 ? fsrc[u * kOzStagePts + 1] : 0.0;
                float d0[kOzDigits], d1[kOzDigits];
                oz_digits(x0, e[u], d0);
                oz_digits(x1, e[u], d1);
                unsigned char* pa = coffa[u] >= 0 ? sst + coffa[u] : nullptr;
                unsigned char* pb = coffb[u] >= 0 ? sst + coffb[u] : nullptr;
#pragma unroll
                for (int s = 0; s < kOzDigits; ++s) {
                    const uint32_t bits = oz_pack2(d0[s], d1[s]);
                    if (pa) *reinterpret_cast<uint32_t*>(pa + soff[s]) = bits;
                    if (pb) *reinterpret_cast<uint32_t*>(pb + soff[s]) = bits;
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[slot]);
        }
        cp_async_wait<0>();                          // no copy may land after the block exits
        if (!ok && lane == 0) fail();
    } else if (warp < kOzSplitWarps) {
        // a split warp without a column
    } else if (warp == kOzMmaWarp) {
        // ------------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc(128, a.nb);
            const uint32_t ring = smem_addr(smem);
            bool ok = true;
            for (int w = 0; w < nwin && ok; ++w) {
                if (w >= 1) {
                    if (!oz_wait(accempty, (unsigned)((w - 1) & 1), abort_flag)) { fail(); break; }
                    tc_fence_after();
                }
                const int st0 = w * kOzWindowStages;
                const int st1 = min(nst, st0 + kOzWindowStages);
                for (int t = st0; t < st1; ++t) {
                    const int slot = t % a.nstage;
                    if (!oz_wait(&full[slot], (unsigned)((t / a.nstage) & 1), abort_flag)) { fail(); ok = false; break; }
                    const uint32_t sa = ring + (uint32_t)(slot * stage_bytes);
                    const uint32_t sb = sa + (uint32_t)a_bytes;
#pragma unroll 1
                    for (int mt = 0; mt < a.nmt; ++mt) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {                       // 16 points per MMA
                            const uint32_t acc = (t > st0 || kk > 0) ? 1u : 0u;
                            mma_bf16(tmem + (uint32_t)(mt * a.nb), sw128_desc(sa + (uint32_t)(mt * 16384) + 32u * kk),
                                     sw128_desc(sb + 32u * kk), idesc, acc);
                        }
                    }
                    mma_commit(&empty[slot]);
                }
                if (ok) mma_commit(accfull);
            }
            // every MMA issued so far has completed once `fin` flips (this wait ignores the abort
            // flag: the tensor memory is released only after them)
            mma_commit(fin);
            if (!mbar_wait(fin, 0u)) {
                fail();
                atomicOr(status, ST_TIMEOUT_MMA);
            }
        }
    } else {
        // ------------------------------------------------------------------ epilogue warps
        // Per accumulation window the entry's share is an integer T60 (about T / 2^60); the 16
        // windows of one exponent window share the scale 2^(E_i + E_j - 52), so their T60 are
        // summed exactly in 128-bit integers and converted to float64 once per exponent window.
        const int quarter = warp & 3;                    // TMEM lanes 32 quarter .. + 31
        const int row = 32 * quarter + lane;             // D line within a tile
        const int s = row & 7;
        double acc[3][kOzMaxJ / 8];
        __int128 iacc[3][kOzMaxJ / 8];
#pragma unroll
        for (int mt = 0; mt < 3; ++mt)
#pragma unroll
            for (int k = 0; k < kOzMaxJ / 8; ++k) {
                acc[mt][k] = 0.0;
                iacc[mt][k] = 0;
            }
        // float64 value of the exact sums of exponent window ew, added to acc
        auto flush = [&](int64_t ew) {
            const int* exw = a.ex + ew * a.r;
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                if (mt >= a.nmt) break;
                const int i = 16 * mt + (row >> 3);
                if (i >= a.q) continue;
                const int ei = __ldg(exw + i);
#pragma unroll
                for (int k = 0; k < kOzMaxJ / 8; ++k) {
                    const int j = 8 * k + s;
                    if (j >= jn) continue;
                    const int ej = __ldg(exw + a.jidx[g][j]);
                    const __int128 v = iacc[mt][k];
                    iacc[mt][k] = 0;
                    if (ei == 2047 || ej == 2047) {
                        acc[mt][k] = __longlong_as_double(0x7FF8000000000000ll);
                        continue;
                    }
                    const long long vh = (long long)(v >> 64);
                    const unsigned long long vl = (unsigned long long)v;
                    // one rounding: directly when v fits in 64 bits (no cancellation of a
                    // negative high word against a large low word), else high and low words
                    const bool fits = (vh == 0 && (long long)vl >= 0) || (vh == -1 && (long long)vl < 0);
                    const double d = fits ? (double)(long long)vl : fma((double)vh, 18446744073709551616.0, (double)vl);
                    acc[mt][k] += ldexp(d, ei + ej - 2096);
                }
            }
        };
        bool ok = true;
        int64_t ew_cur = -1;
        for (int w = 0; w < nwin && ok; ++w) {
            const int64_t ew = (r0 + (int64_t)w * kOzWindowStages * kOzStagePts) / kOzExpPts;
            if (ew != ew_cur) {
                if (ew_cur >= 0) flush(ew_cur);
                ew_cur = ew;
            }
            if (!__all_sync(0xffffffffu, oz_wait(accfull, (unsigned)(w & 1), abort_flag, 256))) { ok = false; break; }
            tc_fence_after();
            const int shl = 17 - 7 * s;
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                if (mt >= a.nmt) break;
                for (int j0 = 0; j0 < jn; j0 += 4) {
                    // 4 columns j (32 accumulator columns) per load; the columns past jn are unused
                    uint32_t r[32];
                    tmem_ld32_nowait(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(mt * a.nb + 8 * j0), r);
                    tmem_wait_ld();
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = j0 + jj;
                        if (j >= jn) break;
                        // this line's digit s against the 8 digits t of column j:
                        //   hi = sum_{t<4} D_st 2^(7 (3 - t)),  lo = sum_{t>=4} D_st 2^(7 (7 - t)),
                        //   share of T >> 60 = hi 2^(17 - 7 s) + lo 2^(-11 - 7 s)
                        long long hi = 0, lo = 0;
#pragma unroll
                        for (int t = 0; t < 4; ++t) hi = hi * 128 + (long long)__float2int_rn(__uint_as_float(r[8 * jj + t]));
#pragma unroll
                        for (int t = 4; t < 8; ++t) lo = lo * 128 + (long long)__float2int_rn(__uint_as_float(r[8 * jj + t]));
                        long long c = shl >= 0 ? hi * (1ll << shl) : (hi >> (-shl));
                        c += lo >> (11 + 7 * s);
                        // the 8 lines of entry (i, j) are 8 consecutive lanes
                        c += __shfl_xor_sync(0xffffffffu, c, 1);
                        c += __shfl_xor_sync(0xffffffffu, c, 2);
                        c += __shfl_xor_sync(0xffffffffu, c, 4);
                        if ((j & 7) == s) iacc[mt][j >> 3] += (__int128)c;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(accempty);
        }
        if (ok && ew_cur >= 0) flush(ew_cur);
        if (!ok) fail();
        // partial sums of this chunk: entry (i, R column jr) -> the S^T S part for S columns, the
        // S^T AS part for AS columns
        if (ok) {
            double* dst = part + (int64_t)blockIdx.x * a.part_stride;
            const int64_t q2 = (int64_t)a.q * a.q;
#pragma unroll
            for (int mt = 0; mt < 3; ++mt) {
                if (mt >= a.nmt) break;
                const int i = 16 * mt + (row >> 3);
                if (i >= a.q) continue;
#pragma unroll
                for (int k = 0; k < kOzMaxJ / 8; ++k) {
                    const int j = 8 * k + s;
                    if (j >= jn) continue;
                    const int jr = a.jidx[g][j];
                    if (jr < a.q) dst[q2 + i + (int64_t)a.q * jr] = acc[mt][k];
                    else dst[i + (int64_t)a.q * (jr - a.q)] = acc[mt][k];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kOzMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

template <int NF>
void launch_oz(const OzArgs& a, dim3 grid, size_t smem, double* part, unsigned* status, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_set{0};   // one bit per device
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        LG_CUDA(cudaFuncSetAttribute(k_gram_oz<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set.fetch_or(bit);
    }
    k_gram_oz<NF><<<grid, kOzThreads, smem, st>>>(a, part, status);
    LG_CHECK_LAUNCH();
}

}  // namespace

bool gram_oz_fits(int q) { return q >= 1 && q <= kOzMaxQ; }

int launch_gram_oz(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int64_t part_doubles,
                   unsigned* status, cudaStream_t st, int* colmax) {
    const int q = S.q();
    LG_REQUIRE(gram_oz_fits(q) && S.t0 == DT_F64 && (S.w[1] + S.w[2] == 0 || S.t12 == DT_F64), LOBPCG_ERR_ARG,
               "tensor-core float64 Gram: float64 basis of at most 48 columns");
    LG_REQUIRE(status != nullptr, LOBPCG_ERR_ARG, "tensor-core float64 Gram needs a status word");
    static thread_local OzArgs a;
    a = OzArgs{};
    auto col = [](const Blocks3& B, int c) {
        int b = 0;
        while (c >= B.w[b]) { c -= B.w[b]; ++b; }
        return static_cast<const double*>(B.p[b]) + (int64_t)c * B.ld;
    };
    a.q = q;
    a.r = AS ? 2 * q : q;
    for (int c = 0; c < q; ++c) {
        a.R[c] = col(S, c);
        if (AS) a.R[q + c] = col(*AS, c);
    }
    a.nmt = (8 * q + 127) / 128;
    // groups of right columns, each with an even share of the S columns and of the AS columns, at
    // most 32 columns, and few enough that the accumulators of every A tile (8 lines per column,
    // rounded up to 32) fit the 512 TMEM columns
    const int jmax = std::min(kOzMaxJ, (512 / a.nmt) / 32 * 32 / 8);
    a.ngroups = (a.r + jmax - 1) / jmax;
    while (a.ngroups <= kOzMaxGroups) {
        bool fits = true;
        for (int g = 0; g < a.ngroups && fits; ++g) {
            const int ns = (q * (g + 1)) / a.ngroups - (q * g) / a.ngroups;
            fits = (AS ? 2 * ns : ns) <= jmax;
        }
        if (fits) break;
        ++a.ngroups;
    }
    LG_REQUIRE(a.ngroups <= kOzMaxGroups, LOBPCG_ERR_ARG, "tensor-core float64 Gram: too many groups");
    int maxjn = 0, maxsplit = 0;
    for (int g = 0; g < a.ngroups; ++g) {
        const int c0 = (q * g) / a.ngroups, c1 = (q * (g + 1)) / a.ngroups;
        int j = 0;
        for (int c = c0; c < c1; ++c) a.jidx[g][j++] = (int16_t)c;
        if (AS)
            for (int c = c0; c < c1; ++c) a.jidx[g][j++] = (int16_t)(q + c);
        a.jn[g] = j;
        maxjn = std::max(maxjn, j);
        maxsplit = std::max(maxsplit, q + (AS ? c1 - c0 : 0));
    }
    a.nb = (8 * maxjn + 31) / 32 * 32;                // the drain reads 32 accumulator columns at once
    a.cpw = (maxsplit + kOzSplitWarps - 1) / kOzSplitWarps;
    const int cols = a.nmt * a.nb;
    a.tmem_cols = 32;
    while (a.tmem_cols < cols) a.tmem_cols *= 2;
    LG_REQUIRE(a.tmem_cols <= 512, LOBPCG_ERR_ARG, "tensor-core float64 Gram: accumulators exceed TMEM");
    const size_t stage_bytes = (size_t)a.nmt * 128 * 128 + (size_t)a.nb * 128;
    const size_t fstage_bytes = (size_t)kOzSplitWarps * a.cpw * kOzStagePts * sizeof(double);
    const size_t fixed = 1024 + 2048;                // alignment slack, barriers and split tables
    // copy ring: about 96 KB of float64 in flight per SM hides the memory latency; two digit stages
    int nf = 16;
    while (nf > 2 && ((size_t)nf * fstage_bytes > 96 * 1024 ||
                      fixed + 2 * stage_bytes + (size_t)nf * fstage_bytes > (size_t)kOzSmemBudget))
        nf /= 2;
    a.nstage = (int)std::min<size_t>(4, ((size_t)kOzSmemBudget - fixed - nf * fstage_bytes) / stage_bytes);
    LG_REQUIRE(a.nstage >= 2, LOBPCG_ERR_ARG, "tensor-core float64 Gram: stage too large");
    // one thread block per SM: row ranges (whole exponent windows) times groups about one wave
    const int64_t q2 = (int64_t)q * q;
    const int64_t nexpw = ceil_div(n, kOzExpPts);
    int nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(kNumSMs / a.ngroups, nexpw));
    // the partial sums, then the exponents (ints), in the scratch
    auto need = [&](int nc) { return (int64_t)nc * 2 * q2 + ceil_div(nexpw * a.r, 2); };
    while (nchunks > 1 && need(nchunks) > part_doubles) --nchunks;
    if (need(nchunks) > part_doubles) return 0;      // scratch too small: the caller falls back
    int* ex = reinterpret_cast<int*>(part + (int64_t)nchunks * 2 * q2);
    a.ex = ex;
    a.n = n;
    a.rows_per_chunk = ceil_div(nexpw, nchunks) * kOzExpPts;
    a.part_stride = 2 * q2;
    const size_t smem = fixed + (size_t)a.nstage * stage_bytes + (size_t)nf * fstage_bytes;
    LG_REQUIRE(smem <= 227 * 1024, LOBPCG_ERR_ARG, "tensor-core float64 Gram: shared memory");
    if (colmax) LG_CUDA(cudaMemsetAsync(colmax, 0, sizeof(int) * a.r, st));
    k_oz_exponents<<<dim3((unsigned)nexpw, (unsigned)((a.r + 7) / 8)), 256, 0, st>>>(a, ex, colmax);
    LG_CHECK_LAUNCH();
    const dim3 grid((unsigned)nchunks, (unsigned)a.ngroups);
    switch (nf) {
        case 16: launch_oz<16>(a, grid, smem, part, status, st); break;
        case 8: launch_oz<8>(a, grid, smem, part, status, st); break;
        case 4: launch_oz<4>(a, grid, smem, part, status, st); break;
        default: launch_oz<2>(a, grid, smem, part, status, st); break;
    }
    return nchunks;
}

}  // namespace lg
