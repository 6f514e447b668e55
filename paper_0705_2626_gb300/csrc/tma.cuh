// Inline PTX for the Tensor Memory Accelerator and shared-memory mbarriers, shared by the
// TMA-staged kernels (k_gram32.cu, k_tsmm.cu, k_tsmm_oz.cu), and the host-side tensor-map encoders.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace lg {

extern thread_local int g_wait_limit;   // run-time poll limit of the stage waits (< 0: default)

// Column blocks of float32 (n rows, w columns, leading dimension ld divisible by 4, 16-byte
// aligned) as a 2-D tensor map with boxes of box_rows x w; rows beyond n read as zeros.  With
// swizzle128 (box_rows = 32: one 128-byte line per column) the box lands in shared memory in the
// 128-byte swizzled layout that the tensor cores read (16-byte chunk c of line r stored at chunk
// c ^ (r mod 8)).
void encode_f32_cols(CUtensorMap* map, const float* p, int64_t n, int w, int64_t ld, int box_rows,
                     bool swizzle128 = false);
// Column blocks of float64 (16-byte aligned, even leading dimension) as a 2-D tensor map with
// boxes of box_rows x w, no swizzle (column c of the box box_rows doubles after column c - 1).
void encode_f64_cols(CUtensorMap* map, const double* p, int64_t n, int w, int64_t ld, int box_rows);

namespace {

constexpr int kSpinLimit = 1 << 22;           // bounded mbarrier waits (polls)

// Polls a stage wait of the TMA-staged float32 kernels may take: the handle's run-time limit
// (lobpcg_set_wait_limit), kSpinLimit unless lowered.  Host side; passed to the kernels.
inline int stage_wait_polls() { return g_wait_limit < 0 ? kSpinLimit : g_wait_limit; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One try_wait on the phase of parity `parity` (the instruction may sleep for a while before it
// reports that the phase is still open).
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, unsigned parity) {
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

// Bounded wait: at most `limit` polls (0: gives up at once).  False if the phase did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit = kSpinLimit) {
#pragma unroll 1
    for (int it = 0; it < limit; ++it)
        if (mbar_poll(bar, parity)) return true;
    return false;
}

// Clean-up after a failed wait: the copies still in flight must land before the block exits.
// The waits of one clean-up share one budget of polls (never the lowered run-time limit).
__device__ __forceinline__ bool mbar_wait_budget(uint64_t* bar, unsigned parity, int& budget) {
#pragma unroll 1
    while (budget > 0) {
        --budget;
        if (mbar_poll(bar, parity)) return true;
    }
    return false;
}

// 2-D tiled copy global -> shared (box = K rows x w columns), completion on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace
}  // namespace lg
