// Tensor-core form of the float32 Gram products of the mixed form (Section 2.2, and
// 17-23): tcgen05 MMAs with operands staged by TMA in shared memory and accumulators in tensor
// memory (TMEM).
//
// The column blocks of one launch are stacked as the lines of a tile: block b occupies lines
// trow[b] .. trow[b] + w[b] - 1 (trow a multiple of 8, unused lines zero), each line holding 32
// consecutive grid points as one 128-byte row in the 128-byte swizzled layout written by the TMA
// copy; L = the stacked lines rounded up to 16.  A pipeline stage holds kTcAtoms such tiles (64
// points), so that the fixed costs of a stage (barrier hand-offs, commits) are shared by 8 MMAs.
//
// Arithmetic (3 x TF32): the tensor cores read a float32 operand as TF32 by dropping its low 13
// mantissa bits (truncation: writing the truncated values back gives bit-identical results), so
// the copy as it landed serves as hi = a with those bits cleared, and the workers store only
// lo = a - hi (exact).  The products are hi*hi + hi*lo + lo*hi; the dropped lo*lo term and the
// TF32 view of lo leave about 2^-21 relative per product.  Two ways to issue them:
//
//  * symmetric form (L <= 128): the lo lines follow the hi lines in the same tile, and one MMA
//    per 8 points, M = 128 (A = lines 0..127) by N = 2L (B = the L hi lines, then the L lo
//    lines), gives HH = hi_i . hi_j in accumulator columns 0..L-1 and H = hi_i . lo_j in columns
//    L..2L-1 for every pair of lines.  The remaining lo_i . hi_j is H transposed: each thread
//    keeps the running sums of H for its row, and at the end they are exchanged through shared
//    memory, so entry (i, j) = sum(HH_ij + H_ij) + sum(H_ji).  Four MMAs per stage;
//  * three-product form (128 < L <= 192): hi tile then lo tile, and three MMAs per 8 points,
//    M = 128 (the left operands, which are the leading lines) by N = L: hi.hi, hi.lo, lo.hi into
//    one accumulator.
//
// The tensor cores keep D in float32 and round each MMA's sum toward zero, so the accumulation
// in TMEM is kept short: D is reset every 128 points (kChunkStages stages) -- 16 MMA steps on
// the dominant hi*hi sum in the symmetric form (the cross products sit in their own columns,
// where the rounding is relative to a 2^-11 smaller sum), 48 in the three-product form.  Worker
// threads read the accumulators with tcgen05.ld and add them into Kahan-compensated float32
// totals in registers; the chunk partials go out as float64 in the layout of the SIMT kernel's,
// and the same fixed-order chunk sums finish the job.
//
// Warp roles (448 threads, one block per SM): warp 0 issues the TMA copies into a ring of
// stages; warp 1 owns the TMEM allocation and one of its threads issues the MMAs and commits
// them to mbarriers; warps 2..13 write the lo lines of each landed stage and drain the
// accumulators.  Shared-memory bandwidth bounds the kernel: per 32 points the copy writes, the
// split reads and writes, and the MMAs read A (128 lines) and B (2L lines) from shared memory.  Two accumulator sets alternate, so the MMAs of one chunk run while the previous
// chunk is drained; the workers drain a finished chunk between stages as soon as its MMAs have
// completed.  Every wait is bounded (status bit ST_TIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "gram_out.cuh"
#include "tma.cuh"

namespace lg {
namespace {

constexpr int kTcWorkWarps = 12;
constexpr int kTcWorkers = 32 * kTcWorkWarps;
constexpr int kTcThreads = 64 + kTcWorkers;       // warp 0: TMA, warp 1: TMEM + MMA, then workers
constexpr int kTcColGroups = kTcWorkWarps / 4;   // workers sharing one TMEM lane quarter
constexpr int kTcMaxL = 192;
constexpr int kTcSymMaxL = 128;
constexpr int kTcMaxBlocks = 6;
constexpr int kTcAtoms = 2;                       // 128-byte swizzle atoms (32 points each) per stage
constexpr int kTcStagePts = 32 * kTcAtoms;
constexpr int kChunkStages = 2;                   // accumulator reset every 128 points
constexpr int kTcSmemBudget = 200 * 1024;
constexpr int kTcCols = 512;                      // TMEM columns: two accumulator sets of 256
constexpr int kWorkerBarrier = 1;                 // named barrier of the worker warps

struct GtcArgs {
    CUtensorMap map[kTcMaxBlocks];
    int nblk;
    int trow[kTcMaxBlocks];
    unsigned tx;                  // bytes landing per stage
    int L;                        // stacked lines, rounded up to 16
    int lo_lines;                 // lo line k sits lo_lines lines after hi line k
    int stage_lines;              // lines per stage (hi, lo and zero padding)
    int rows;                     // D rows (lines) that are drained
    int nstage;
    int64_t rows_per_chunk, part_stride;
    int nout;
    G32Out out[2];
    int16_t lmap[kTcMaxL];        // line -> staged column (-1: padding)
};

// ---- tcgen05 / TMEM primitives (inline PTX) ---------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait that also gives up as soon as another role has flagged a failure.  The worker
// warps sleep in try_wait; the single-thread TMA and MMA roles poll with test_wait, which reacts
// to the phase change sooner.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, unsigned parity, volatile int* abort_flag) {
#pragma unroll 1
    for (int it = 0; it < kSpinLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ bool mbar_poll_or_abort(uint64_t* bar, unsigned parity, volatile int* abort_flag) {
#pragma unroll 1
    for (int it = 0; it < 16 * kSpinLimit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    return false;
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzled layout, 8-line
// groups 1024 bytes apart (stride byte offset), descriptor version 1 (bits 46-48 = 0b001),
// swizzle mode 2 (128 B) in bits 61-63; the leading byte offset is unused for this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::tf32: D float32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns: thread t of the warp gets lane (lane field + t).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ float4 tf32_hi(float4 v) {
    auto h = [](float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); };
    return make_float4(h(v.x), h(v.y), h(v.z), h(v.w));
}

// SLOTS: 16-column slices of D per worker thread (ceil(L / 16 / kTcColGroups)); SYM: the
// symmetric form (L <= 128), else the three-product form.
template <int SLOTS, bool SYM>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const __grid_constant__ GtcArgs a, int64_t n, double* __restrict__ part, unsigned* status) {
    extern __shared__ unsigned char smem_raw[];
    // swizzled operand tiles must start on a 1024-byte boundary
    unsigned char* smem = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    const int atom_bytes = a.stage_lines * 128;                  // one 32-point tile
    const int stage_bytes = kTcAtoms * atom_bytes;
    const int lo_bytes = a.lo_lines * 128;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)a.nstage * stage_bytes);
    uint64_t* ready = full + a.nstage;
    uint64_t* empty = ready + a.nstage;
    uint64_t* accfull = empty + a.nstage;                         // two accumulator sets
    uint64_t* accempty = accfull + 2;
    uint64_t* fin = accempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* issued_out = reinterpret_cast<volatile int*>(tslot + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = blockIdx.x * a.rows_per_chunk;
    const int64_t r1 = min(n, r0 + a.rows_per_chunk);
    const int nst = r1 > r0 ? (int)((r1 - r0 + kTcStagePts - 1) / kTcStagePts) : 0;

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&ready[s], kTcWorkers);
            mbar_init(&empty[s], 1);
        }
        for (int c = 0; c < 2; ++c) {
            mbar_init(&accfull[c], 1);
            mbar_init(&accempty[c], kTcWorkers);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        *issued_out = 0;
        mbar_fence_init();
    }
    // padding lines of every stage stay zero (the copies and the split write the data lines only)
    {
        uint4* z = reinterpret_cast<uint4*>(smem);
        const int nz = a.nstage * stage_bytes / 16;
        for (int i = tid; i < nz; i += kTcThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr int kSet = kTcCols / 2;                              // columns per accumulator set
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
    };

    // per-worker state (registers: only the workers touch it)
    const bool worker = warp >= 2;
    const int quarter = warp & 3;                                  // TMEM lanes 32*quarter .. +31
    const int cgrp = worker ? (warp - 2) >> 2 : 0;
    const bool warp_rows = worker && 32 * quarter < a.rows;
    const int nslices = a.L / 16;
    float tot[SLOTS][16];
    __nv_bfloat162 cmpb[SLOTS][8];
    float ht[SYM ? SLOTS : 1][16];                                 // running sums of H (symmetric form)
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
#pragma unroll
        for (int e = 0; e < 16; ++e) tot[k][e] = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) cmpb[k][e] = __floats2bfloat162_rn(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < (SYM ? SLOTS : 1); ++k)
#pragma unroll
        for (int e = 0; e < 16; ++e) ht[k][e] = 0.f;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int t = 0, s = 0, u = 0; t < nst; ++t) {
                if (t >= a.nstage && !mbar_poll_or_abort(&empty[s], (unsigned)((u - 1) & 1), abort_flag)) {
                    fail();
                    break;
                }
                unsigned char* st_base = smem + (size_t)s * stage_bytes;
                mbar_expect_tx(&full[s], a.tx);
                for (int at = 0; at < kTcAtoms; ++at)
                    for (int b = 0; b < a.nblk; ++b)
                        tma_load_2d(st_base + at * atom_bytes + a.trow[b] * 128, &a.map[b],
                                    (int)(r0 + (int64_t)t * kTcStagePts + 32 * at), 0, &full[s]);
                issued = t + 1;
                if (++s == a.nstage) {
                    s = 0;
                    ++u;
                }
            }
            *issued_out = issued;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tf32_idesc(128, SYM ? 2 * a.L : a.L);
            const uint32_t ring = smem_addr(smem);
            for (int t = 0, s = 0, u = 0; t < nst; ++t) {
                const int c = t / kChunkStages;
                const bool first = t % kChunkStages == 0;
                if (first && c >= 2) {
                    if (!mbar_poll_or_abort(&accempty[c & 1], (unsigned)(((c - 2) >> 1) & 1), abort_flag)) {
                        fail();
                        break;
                    }
                    tc_fence_after();
                }
                // the split's writes reach the tensor cores' (async) proxy through the workers'
                // fence.proxy.async before their arrival on ready[s]
                if (!mbar_poll_or_abort(&ready[s], (unsigned)(u & 1), abort_flag)) {
                    fail();
                    break;
                }
                const uint32_t d = tmem + (uint32_t)((c & 1) * kSet);
#pragma unroll
                for (int at = 0; at < kTcAtoms; ++at) {
                    const uint32_t hi = ring + (uint32_t)(s * stage_bytes + at * atom_bytes);
                    const uint32_t lo = hi + (uint32_t)lo_bytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {                // 8 points (32 bytes) per MMA
                        const uint64_t dh = sw128_desc(hi + 32u * kk);
                        const uint32_t acc = (first && at == 0 && kk == 0) ? 0u : 1u;
                        if constexpr (SYM) {
                            mma_tf32(d, dh, dh, idesc, acc);        // B = hi lines then lo lines
                        } else {
                            const uint64_t dl = sw128_desc(lo + 32u * kk);
                            mma_tf32(d, dh, dh, idesc, acc);
                            mma_tf32(d, dh, dl, idesc, 1u);
                            mma_tf32(d, dl, dh, idesc, 1u);
                        }
                    }
                }
                mma_commit(&empty[s]);
                if (t % kChunkStages == kChunkStages - 1 || t == nst - 1) mma_commit(&accfull[c & 1]);
                if (++s == a.nstage) {
                    s = 0;
                    ++u;
                }
            }
            // every MMA issued so far has completed once `fin` flips.  This wait ignores the abort
            // flag: the accumulators are deallocated and the stage ring released only after the
            // MMAs issued before an abort have finished (bounded; ST_TIMEOUT_MMA if even that
            // wait gives up).
            mma_commit(fin);
            if (!mbar_wait(fin, 0u)) {
                fail();
                atomicOr(status, ST_TIMEOUT_MMA);
            }
        }
    } else {
        const int wt = tid - 64;
        // add the accumulators of chunk c into the totals (the chunk's MMAs have completed)
        auto drain_now = [&](int c) {
            tc_fence_after();
            if (warp_rows) {
#pragma unroll
                for (int k = 0; k < SLOTS; ++k) {
                    const int sl = cgrp + kTcColGroups * k;
                    if (sl < nslices) {
#pragma unroll
                        for (int hv = 0; hv < 2; ++hv) {
                            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) +
                                                (uint32_t)((c & 1) * kSet + 16 * sl + 8 * hv);
                            float v[8];
                            tmem_ld8(ta, v);
                            if constexpr (SYM) {
                                float x[8];
                                tmem_ld8(ta + (uint32_t)a.L, x);     // H = hi . lo columns
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    v[e] = __fadd_rn(v[e], x[e]);
                                    ht[k][8 * hv + e] = __fadd_rn(ht[k][8 * hv + e], x[e]);
                                }
                            }
#pragma unroll
                            for (int e = 0; e < 8; e += 2) {
                                const int ee = 8 * hv + e;
                                float c2[2] = {__low2float(cmpb[k][ee / 2]), __high2float(cmpb[k][ee / 2])};
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    const float y = __fsub_rn(v[e + h], c2[h]);
                                    const float tt = __fadd_rn(tot[k][ee + h], y);
                                    c2[h] = __fsub_rn(__fsub_rn(tt, tot[k][ee + h]), y);
                                    tot[k][ee + h] = tt;
                                }
                                cmpb[k][ee / 2] = __floats2bfloat162_rn(c2[0], c2[1]);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[c & 1]);
        };
        // warp-uniform non-blocking test: true once every lane has observed the phase (each
        // lane's own test orders its later reads after the phase)
        auto poll = [&](uint64_t* bar, unsigned parity) { return __all_sync(0xffffffffu, mbar_test(bar, parity)); };
        // bounded wait with a warp-uniform outcome (the drain's tcgen05.ld needs the whole warp)
        auto wait_all = [&](uint64_t* bar, unsigned parity) {
            return __all_sync(0xffffffffu, mbar_wait_or_abort(bar, parity, abort_flag));
        };
        bool ok = true;
        int pending = -1;                                          // finished chunk not yet drained
        const int nf4a = a.L * 8;                                  // float4s of the data lines of a tile
        const int nf4 = kTcAtoms * nf4a;
        for (int t = 0; t < nst && ok; ++t) {
            const int s = t % a.nstage, u = t / a.nstage;
            // one non-blocking look per stage for a finished chunk, then sleep in try_wait until
            // the stage lands (spinning would take issue slots from the MMA and TMA threads)
            if (pending >= 0 && poll(&accfull[pending & 1], (unsigned)((pending >> 1) & 1))) {
                drain_now(pending);
                pending = -1;
            }
            if (!wait_all(&full[s], (unsigned)(u & 1))) {
                ok = false;
                break;
            }
            for (int f = wt; f < nf4; f += kTcWorkers) {
                const int at = f / nf4a, g = f - at * nf4a;
                unsigned char* tile = smem + (size_t)s * stage_bytes + (size_t)at * atom_bytes;
                float4* hi = reinterpret_cast<float4*>(tile);
                float4* lo = reinterpret_cast<float4*>(tile + lo_bytes);
                const float4 v = hi[g];
                const float4 h = tf32_hi(v);
                lo[g] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
            }
            fence_proxy_async();
            mbar_arrive(&ready[s]);
            if (t % kChunkStages == kChunkStages - 1 || t == nst - 1) {
                // this stage closes chunk t / kChunkStages; the previous one must be drained
                // before the MMAs of the chunk after this one reuse its accumulators
                if (pending >= 0) {
                    if (!wait_all(&accfull[pending & 1], (unsigned)((pending >> 1) & 1))) {
                        ok = false;
                        break;
                    }
                    drain_now(pending);
                }
                pending = t / kChunkStages;
            }
        }
        if (ok && pending >= 0) {
            if (wait_all(&accfull[pending & 1], (unsigned)((pending >> 1) & 1)))
                drain_now(pending);
            else
                ok = false;
        }
        if (!ok) fail();
    }

    tc_fence_before();
    __syncthreads();
    const bool aborted = *abort_flag != 0;
    if (aborted && tid == 0) {
        // let the copies still in flight land before the block exits (only the last nstage
        // issued can be; each wait bounded)
        const int issued = *issued_out;
        for (int t = max(0, issued - a.nstage); t < issued; ++t)
            for (int it = 0; it < kSpinLimit && !mbar_try(&full[t % a.nstage], (unsigned)((t / a.nstage) & 1)); ++it) {
            }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
    if (aborted || !worker) return;

    // symmetric form: the H sums of every line, transposed through shared memory (the stage
    // ring is idle now: every copy has landed and every MMA has completed)
    const int row = 32 * quarter + lane;
    float* hs = reinterpret_cast<float*>(smem);                   // L x L, hs[i * L + j] = sum H_ij
    if constexpr (SYM) {
        if (warp_rows && row < a.L) {
#pragma unroll
            for (int k = 0; k < SLOTS; ++k) {
                const int sl = cgrp + kTcColGroups * k;
                if (sl < nslices)
#pragma unroll
                    for (int e = 0; e < 16; ++e) hs[row * a.L + 16 * sl + e] = ht[k][e];
            }
        }
        asm volatile("bar.sync %0, %1;" ::"n"(kWorkerBarrier), "n"(kTcWorkers) : "memory");
    }
    if (!warp_rows || row >= a.rows) return;
    const int li = a.lmap[row];
    if (li < 0) return;
    double* dst = part + blockIdx.x * a.part_stride;
#pragma unroll
    for (int k = 0; k < SLOTS; ++k) {
        const int sl = cgrp + kTcColGroups * k;
        if (sl >= nslices) continue;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int col = 16 * sl + e;
            const int lj = a.lmap[col];
            if (lj < 0) continue;
            const float c = (e & 1) ? __high2float(cmpb[k][e / 2]) : __low2float(cmpb[k][e / 2]);
            double val = (double)tot[k][e] - (double)c;
            if constexpr (SYM) val += (double)hs[col * a.L + row];   // sum of lo_i . hi_j
            for (int oi = 0; oi < a.nout; ++oi) {
                const G32Out& o = a.out[oi];
                const int i = li - o.lbase, j = lj - o.rbase;
                if (g32_need(o, i, j)) dst[o.off + i + (int64_t)o.ld * j] = val;
            }
        }
    }
}

template <int SLOTS, bool SYM>
void launch_tc(const GtcArgs& a, int nchunks, size_t smem, int64_t n, double* part, unsigned* status,
               cudaStream_t st) {
    static std::atomic<unsigned long long> attr_set{0};   // one bit per device
    int dev = 0;
    LG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set.load() & bit)) {
        LG_CUDA(cudaFuncSetAttribute(k_gram_tc<SLOTS, SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set.fetch_or(bit);
    }
    k_gram_tc<SLOTS, SYM><<<(unsigned)nchunks, kTcThreads, smem, st>>>(a, n, part, status);
    LG_CHECK_LAUNCH();
}

}  // namespace

bool launch_gram_tc(const G32Block* blk, int nblk, const G32Out* out, int nout, int64_t part_stride, int64_t n,
                    int64_t ld, int nchunks, double* part, unsigned* status, int mode, cudaStream_t st) {
    if (mode == GRAM_TC_NEVER) return false;
    static thread_local GtcArgs a;    // ~1 KB of tensor maps: keep it off the stack
    a = GtcArgs{};
    for (int i = 0; i < kTcMaxL; ++i) a.lmap[i] = -1;
    // stack the blocks as lines, each block on an 8-line boundary
    int line = 0;
    a.nblk = 0;
    for (int b = 0; b < nblk; ++b) {
        if (blk[b].w <= 0) continue;
        if (a.nblk >= kTcMaxBlocks) return false;
        line = (line + 7) / 8 * 8;
        if (line + blk[b].w > kTcMaxL) return false;
        a.trow[a.nblk] = line;
        for (int c = 0; c < blk[b].w; ++c) a.lmap[line + c] = (int16_t)(blk[b].coff + c);
        line += blk[b].w;
        ++a.nblk;
    }
    if (a.nblk == 0) return false;
    a.L = std::max(16, (line + 15) / 16 * 16);
    if (a.L > kTcMaxL || (mode == GRAM_TC_WIDE && a.L <= kGramTcWide)) return false;
    const bool sym = a.L <= kTcSymMaxL;
    auto line_of = [&](int staged) {
        for (int r = 0; r < kTcMaxL; ++r)
            if (a.lmap[r] == staged) return r;
        return -1;
    };
    // every needed entry (i, j) must come from D row line_of(i), column line_of(j); the rows are
    // the A operand's lines 0..127
    int qa = 0;
    for (int oi = 0; oi < nout; ++oi) {
        const G32Out& o = out[oi];
        for (int i = 0; i < o.rows; ++i) {
            bool used = false;
            for (int j = 0; j < o.cols && !used; ++j) used = g32_need(o, i, j);
            if (!used) continue;
            const int r = line_of(o.lbase + i);
            if (r < 0 || r >= 128) return false;
            qa = std::max(qa, r + 1);
        }
        for (int j = 0; j < o.cols; ++j)
            if (line_of(o.rbase + j) < 0) return false;
    }
    a.rows = sym ? a.L : qa;                 // the symmetric form needs the H sums of every line
    a.lo_lines = sym ? a.L : std::max(128, a.L);
    a.stage_lines = sym ? std::max(128, 2 * a.L) : 2 * a.lo_lines;
    a.nout = nout;
    for (int oi = 0; oi < nout; ++oi) a.out[oi] = out[oi];
    a.part_stride = part_stride;
    a.rows_per_chunk = ceil_div(ceil_div(n, nchunks), 128) * 128;
    const int stage_bytes = kTcAtoms * a.stage_lines * 128;
    a.nstage = std::max(2, std::min(8, kTcSmemBudget / stage_bytes));
    a.tx = 0;
    int k = 0;
    for (int b = 0; b < nblk; ++b) {
        if (blk[b].w <= 0) continue;
        encode_f32_cols(&a.map[k], blk[b].p, n, blk[b].w, ld, 32, true);
        a.tx += (unsigned)(kTcStagePts * blk[b].w * sizeof(float));
        ++k;
    }
    const size_t smem = 1024 + (size_t)a.nstage * stage_bytes + (3 * (size_t)a.nstage + 5) * 8 + 16;
    LG_REQUIRE(smem <= 227 * 1024, LOBPCG_ERR_ARG, "tensor-core Gram stage too large");
    // the transposed H sums reuse the stage ring
    LG_REQUIRE(!sym || (size_t)a.L * a.L * sizeof(float) <= (size_t)a.nstage * stage_bytes, LOBPCG_ERR_ARG,
               "tensor-core Gram exchange buffer too small");
    const int slots = (a.L / 16 + kTcColGroups - 1) / kTcColGroups;
    if (sym) {
        switch (slots) {
            case 1: launch_tc<1, true>(a, nchunks, smem, n, part, status, st); break;
            case 2: launch_tc<2, true>(a, nchunks, smem, n, part, status, st); break;
            default: launch_tc<3, true>(a, nchunks, smem, n, part, status, st); break;
        }
    } else {
        if (slots <= 3) launch_tc<3, false>(a, nchunks, smem, n, part, status, st);
        else launch_tc<4, false>(a, nchunks, smem, n, part, status, st);
    }
    return true;
}

}  // namespace lg
