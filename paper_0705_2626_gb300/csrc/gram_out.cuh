// Output maps of the tall-skinny float32 Gram kernels (the SIMT tiles in k_gram32.cu and the
// tensor-core form in k_gram_tc.cu): which entries of which small matrix a launch produces, and
// where its per-chunk partial sums go.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lg {

enum G32Mode : int { G32_ALL = 0, G32_UPPER = 1, G32_MXA = 2, G32_MXB = 3 };

// One output matrix: entry (i, j) = column (lbase + i) . column (rbase + j) of the staged
// columns, stored at part[chunk * part_stride + off + i + ld * j] when `need` holds.
struct G32Out {
    int64_t off;
    int ld;
    int lbase, rbase;
    int rows, cols;
    int mode;
    int w0, w1;       // widths of the X and W blocks (mixed-form predicates)
};

// A float32 column block (n rows, leading dimension shared by all blocks of a launch) and the
// index of its first column among the staged columns.
struct G32Block {
    const float* p;
    int w;
    int coff;
};

__host__ __device__ inline int blk3(int i, int w0, int w1) { return i < w0 ? 0 : (i < w0 + w1 ? 1 : 2); }

__host__ __device__ inline bool g32_need(const G32Out& o, int i, int j) {
    if (i < 0 || j < 0 || i >= o.rows || j >= o.cols) return false;
    switch (o.mode) {
        case G32_UPPER: return i <= j;
        // S^T T of the residual form: every row against an X column, and the upper block
        // triangle of the W / P part (diagonal blocks in full)
        case G32_MXA: return j < o.w0 || (i >= o.w0 && blk3(i, o.w0, o.w1) <= blk3(j, o.w0, o.w1));
        // S^T S upper triangle outside the X^T X block (that block is double-float)
        case G32_MXB: return i <= j && j >= o.w0;
        default: return true;
    }
}

// When to use the tensor-core form of the float32 products.
enum GramTc : int { GRAM_TC_NEVER = 0, GRAM_TC_WIDE = 1, GRAM_TC_ALWAYS = 2 };
// Stacks wider than this many columns go to the tensor cores under GRAM_TC_WIDE: an MMA costs
// about the same for any N, so narrow stacks are cheaper on the SIMT tiles.
constexpr int kGramTcWide = 64;

// Tensor-core form of the float32 products: the same outputs and partial-sum layout as the SIMT
// tiles, over `nchunks` row chunks of ceil(ceil(n / nchunks) / 128) * 128 rows.  Returns false
// without launching when the blocks do not fit its tile, or under GRAM_TC_WIDE when the stack is
// narrow (then the caller runs the SIMT kernel).
bool launch_gram_tc(const G32Block* blk, int nblk, const G32Out* out, int nout, int64_t part_stride, int64_t n,
                    int64_t ld, int nchunks, double* part, unsigned* status, int mode, cudaStream_t st);

}  // namespace lg
