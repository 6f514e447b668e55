// Tall-skinny block kernels of one LOBPCG iteration (B = I):
//   random initial block (Algorithm input X, SplitMix64 counter generator),
//   residuals and their norms (Section 2.2),
//   Gram matrices [X W_J P_J]^T [AX AW_J AP_J] and [X W_J P_J]^T [X W_J P_J] (the Gram matrices of the Rayleigh-Ritz basis,
//   and the Cholesky Gram matrices of the orthonormalisations of X, W and P),
//   multiplication by the inverse Cholesky factor (the orthonormalisations of X, W and P),
//   the Ritz update of P, AP, X, AX (the Ritz update).
// Blocks are float64 in the FP64 form; in the mixed form X and AX stay float64 and the W / P
// family is float32 (products in float32, sums compensated).  Reductions over the n grid points
// are deterministic: per-thread-block partial sums land in scratch memory and are added in a
// fixed order by a second kernel, so repeated runs are bit-identical.
#include <type_traits>

#include "common.cuh"
#include "dtype.cuh"

namespace lg {
namespace {

// ------------------------------------------------------------------ SplitMix64
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_random_block(uint64_t seed, int64_t n, int m, double* __restrict__ X, int64_t ldx) {
    const int64_t total = n * m;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / n, p = t - j * n;
        const uint64_t z = splitmix64_out(seed, (uint64_t)t);
        X[j * ldx + p] = (double)(z >> 11) * 0x1p-52 - 1.0;   // 2 * (z >> 11) * 2^-53 - 1, exact
    }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the thread block in a fixed order; result valid in thread 0.
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        s = lane < nw ? red[lane] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

constexpr int kResThreads = 256;

// W[:, t] = AX[:, j] - lambda_j X[:, j] in float64 (stored as TW), j = cols[t]; the norms come
// from the float64 values.
template <typename TW>
__global__ void __launch_bounds__(kResThreads)
    k_residual(int64_t n, int64_t rows_per_chunk, ColList cols, const double* __restrict__ X,
               const double* __restrict__ AX, int64_t ld, const double* __restrict__ lam,
               TW* __restrict__ W, int64_t ldw, double* __restrict__ partial, int nchunks) {
    __shared__ double red[32];
    const int t = blockIdx.y;
    const int j = cols.idx[t];
    const double lj = lam[j];
    const int64_t r0 = blockIdx.x * rows_per_chunk;
    const int64_t r1 = min(n, r0 + rows_per_chunk);
    const double* xc = X + (int64_t)j * ld;
    const double* ac = AX + (int64_t)j * ld;
    TW* wc = W ? W + (int64_t)t * ldw : nullptr;
    double acc = 0.0;
    for (int64_t p = r0 + threadIdx.x; p < r1; p += blockDim.x) {
        const double w = fma(-lj, __ldg(xc + p), __ldg(ac + p));
        if (wc) st_as(wc + p, w);
        acc = fma(w, w, acc);
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[(int64_t)t * nchunks + blockIdx.x] = s;
}

__global__ void k_norms_finalize(int nchunks, const double* __restrict__ partial,
                                 double* __restrict__ norms) {
    const int t = blockIdx.x;
    double s = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += 32) s += partial[(int64_t)t * nchunks + c];
    s = warp_sum(s);
    if (threadIdx.x == 0) norms[t] = sqrt(s);
}

// ------------------------------------------------------------------ Gram
constexpr int kTM = 4;    // each thread owns a kTM x kTM tile of the output
constexpr int kCG = 4;    // output columns per thread of the update-type kernels

template <typename T0, typename T12, typename C>
__device__ __forceinline__ C load_col(const Blocks3& B, int c, int64_t p) {
    if (c < B.w[0]) return (C)ld_as(static_cast<const T0*>(B.p[0]) + (int64_t)c * B.ld + p);
    c -= B.w[0];
    if (c < B.w[1]) return (C)ld_as(static_cast<const T12*>(B.p[1]) + (int64_t)c * B.ld + p);
    c -= B.w[1];
    return (C)ld_as(static_cast<const T12*>(B.p[2]) + (int64_t)c * B.ld + p);
}

__host__ __device__ inline int block_of(const Blocks3& B, int c) {
    return c < B.w[0] ? 0 : (c < B.w[0] + B.w[1] ? 1 : 2);
}

// Output tile (ti, tj) of S^T AS is needed when it holds an entry (i, j) with
// block(i) <= block(j): the upper block triangle of the Gram blocks as printed, diagonal blocks in full.
// First tile column of the needed A tiles in tile row ti: the tile holding the first column of
// the block of column ti * kTM (block(j) >= block(i) from there on).
__host__ __device__ inline int a_tile_first(const Blocks3& B, int ti) {
    const int b = block_of(B, ti * kTM);
    const int c0 = b == 0 ? 0 : (b == 1 ? B.w[0] : B.w[0] + B.w[1]);
    return c0 / kTM;
}

constexpr int kGramMaxThreads = 768;            // threads of one Gram block
constexpr int kGramSmemMax = 200 * 1024;        // stage buffers and group reduction
constexpr int kGramSmemPair = 96 * 1024;        // narrow bases: two blocks per SM

struct GramShape {
    int ntA, ntB, nt;   // needed A tiles, upper B tiles, all tiles
    int tpb, ngroups;   // tiles per thread block, thread blocks (tile groups) per row range
    int ks, gk;         // row groups per tile, rows per stage
};

__host__ __device__ inline GramShape gram_shape(const Blocks3& S, bool with_a, int elt) {
    const int q = S.q();
    const int T = (q + kTM - 1) / kTM;
    GramShape g;
    g.ntA = 0;
    if (with_a)
        for (int ti = 0; ti < T; ++ti) g.ntA += T - a_tile_first(S, ti);
    g.ntB = T * (T + 1) / 2;
    g.nt = g.ntA + g.ntB;
    // wide bases: the tiles are split over ngroups thread blocks that share a row range
    g.ngroups = (g.nt + kGramMaxThreads - 1) / kGramMaxThreads;
    g.tpb = (g.nt + g.ngroups - 1) / g.ngroups;
    // narrow bases: several row groups per tile, about 256 threads, and at most 96 KB of shared
    // memory so that two blocks share an SM (one stages its rows while the other computes)
    g.ks = max(1, min(64, 256 / g.tpb));
    const int arrays = with_a ? 2 : 1;
    while (g.ks > 1 && max(arrays * 16 * g.ks * (T * kTM + 1) * elt, g.ks * g.tpb * 16 * 8) > kGramSmemPair) --g.ks;
    g.gk = 16 * g.ks;
    return g;
}

__host__ __device__ inline size_t gram_smem_bytes(const GramShape& g, int q, bool with_a, int elt) {
    const int T = (q + kTM - 1) / kTM;
    const size_t stage = (size_t)(with_a ? 2 : 1) * g.gk * (T * kTM + 1) * elt;
    const size_t red = g.ks > 1 ? (size_t)g.ks * g.tpb * 16 * sizeof(double) : 0;
    return stage > red ? stage : red;
}

// Partial sums over one row range per thread block of the needed tiles of S^T AS ("A") and of
// the upper tiles of S^T S ("B").  Tiles are numbered A first, then B, each row-major; thread
// block (r, y) takes the tiles y * tpb .. y * tpb + tpb - 1 of row range r.  Thread t works on
// its block's tile t % tpb for the rows of each shared-memory stage congruent to t / tpb modulo
// ks (16 rows per stage and thread); the ks row groups are added in a fixed order at the end.
// A warp shares ti (broadcast reads of S).  C = double: float64 products and sums.  C = float:
// float32 products summed over the 16 rows of a stage, stage sums added with Kahan's
// compensated summation, the result rounded to float64.
template <typename T0, typename T12, typename C>
__global__ void __launch_bounds__(kGramMaxThreads)
    k_gram(int64_t n, int64_t rows_per_part, Blocks3 S, Blocks3 AS, int with_a,
           double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sm = reinterpret_cast<C*>(sm_raw);
    const int q = S.q();
    const int T = (q + kTM - 1) / kTM;
    const GramShape gs = gram_shape(S, with_a != 0, (int)sizeof(C));
    const int tpb = gs.tpb;
    const int ldsm = T * kTM + 1;                 // odd row length: conflict-free stores
    C* sS = sm;                                   // [gk][ldsm]
    C* sA = sm + gs.gk * ldsm;                    // [gk][ldsm]
    const int tl = threadIdx.x % tpb;
    const int grp = threadIdx.x / tpb;
    const int tile = blockIdx.y * tpb + tl;
    const bool active = grp < gs.ks && tile < gs.nt;
    const bool isA = tile < gs.ntA;
    int ti = 0, tj = 0;
    if (isA) {
        int u = tile;                             // u-th needed A tile, row-major
        for (int r = 0; r < T; ++r) {
            const int first = a_tile_first(S, r), cnt = T - first;
            if (u < cnt) { ti = r; tj = first + u; break; }
            u -= cnt;
        }
    } else if (tile < gs.nt) {
        int u = tile - gs.ntA;                    // upper B tiles ti <= tj, row-major
        while (u >= T - ti) { u -= T - ti; ++ti; }
        tj = ti + u;
    }
    C acc[kTM][kTM];          // running sums (float64), or the current stage's sums (float32)
    C cmp[kTM][kTM];          // Kahan compensation (float32 only)
    C tot[kTM][kTM];          // compensated running sums (float32 only)
#pragma unroll
    for (int a = 0; a < kTM; ++a)
#pragma unroll
        for (int b = 0; b < kTM; ++b) acc[a][b] = cmp[a][b] = tot[a][b] = C(0);

    const int64_t r0 = blockIdx.x * rows_per_part;
    const int64_t r1 = min(n, r0 + rows_per_part);
    const C* rhs = isA ? sA : sS;
    constexpr int kLoadBatch = 4;                 // loads in flight per thread while staging
    const int nstage_elems = gs.gk * T * kTM;
    for (int64_t base = r0; base < r1; base += gs.gk) {
        for (int arr = 0; arr < (with_a ? 2 : 1); ++arr) {
            const Blocks3& B = arr ? AS : S;
            C* dst = arr ? sA : sS;
            for (int e0 = threadIdx.x; e0 < nstage_elems; e0 += kLoadBatch * blockDim.x) {
                C v[kLoadBatch];
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u) {
                    const int e = e0 + u * blockDim.x;
                    const int c = e / gs.gk, k = e - c * gs.gk;
                    const int64_t p = base + k;
                    v[u] = (e < nstage_elems && c < q && p < r1) ? load_col<T0, T12, C>(B, c, p) : C(0);
                }
#pragma unroll
                for (int u = 0; u < kLoadBatch; ++u) {
                    const int e = e0 + u * blockDim.x;
                    if (e < nstage_elems) {
                        const int c = e / gs.gk, k = e - c * gs.gk;
                        dst[k * ldsm + c] = v[u];
                    }
                }
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int k = grp; k < gs.gk; k += gs.ks) {
                C a[kTM], b[kTM];
#pragma unroll
                for (int u = 0; u < kTM; ++u) {
                    a[u] = sS[k * ldsm + ti * kTM + u];
                    b[u] = rhs[k * ldsm + tj * kTM + u];
                }
#pragma unroll
                for (int u = 0; u < kTM; ++u)
#pragma unroll
                    for (int v = 0; v < kTM; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
            if constexpr (std::is_same<C, float>::value) {
#pragma unroll
                for (int u = 0; u < kTM; ++u)
#pragma unroll
                    for (int v = 0; v < kTM; ++v) {
                        const C y = acc[u][v] - cmp[u][v];
                        const C t = tot[u][v] + y;
                        cmp[u][v] = (t - tot[u][v]) - y;
                        tot[u][v] = t;
                        acc[u][v] = C(0);
                    }
            }
        }
        __syncthreads();
    }
    double res[kTM][kTM];
#pragma unroll
    for (int u = 0; u < kTM; ++u)
#pragma unroll
        for (int v = 0; v < kTM; ++v) {
            if constexpr (std::is_same<C, float>::value) res[u][v] = (double)tot[u][v] - (double)cmp[u][v];
            else res[u][v] = acc[u][v];
        }
    // add the row groups in order 0, 1, ..., ks-1 (the stage buffers are free now)
    if (gs.ks > 1) {
        double* red = reinterpret_cast<double*>(sm_raw);   // [ks][tpb][16]
        if (active)
#pragma unroll
            for (int u = 0; u < kTM; ++u)
#pragma unroll
                for (int v = 0; v < kTM; ++v) red[((int64_t)grp * tpb + tl) * 16 + u * kTM + v] = res[u][v];
        __syncthreads();
        if (grp == 0 && active) {
#pragma unroll
            for (int u = 0; u < kTM; ++u)
#pragma unroll
                for (int v = 0; v < kTM; ++v) {
                    double sum = red[(int64_t)tl * 16 + u * kTM + v];
                    for (int g = 1; g < gs.ks; ++g) sum += red[((int64_t)g * tpb + tl) * 16 + u * kTM + v];
                    res[u][v] = sum;
                }
        }
    }
    if (grp != 0 || !active) return;
    double* out = part + (int64_t)blockIdx.x * 2 * q * q + (isA ? 0 : (int64_t)q * q);
#pragma unroll
    for (int u = 0; u < kTM; ++u)
#pragma unroll
        for (int v = 0; v < kTM; ++v) {
            const int i = ti * kTM + u, j = tj * kTM + v;
            if (i < q && j < q) out[i + (int64_t)q * j] = res[u][v];
        }
}

// gramA / gramB of the mixed form in residual form (S = [X W P], T = [R AW AP], R = AX - X Lambda)
// from the partial sums of S^T T (entries (i, j) with column j in X or 1 <= block(i) <= block(j))
// and S^T S (i <= j): X^T AX = (X^T X) Lambda + X^T R symmetrised,
// (AX)^T s_j = Lambda X^T s_j + R^T s_j, and the W / P part as in the float64 form.  One warp per
// pair i <= j.
__global__ void k_gram_finalize_mx(int q, int nparts, const double* __restrict__ part,
                                   double* __restrict__ gA, double* __restrict__ gB,
                                   const double* __restrict__ lam, Blocks3 W) {
    const int64_t pair = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t npairs = (int64_t)q * (q + 1) / 2;
    if (pair >= npairs) return;
    int j = 0;
    int64_t u = pair;
    while (u >= j + 1) { u -= j + 1; ++j; }
    const int i = (int)u;
    const int bi = block_of(W, i), bj = block_of(W, j);
    const int64_t q2 = (int64_t)q * q;
    // entries written by k_gram_mx: (i, j) when column j is in X or 1 <= block(i) <= block(j)
    const bool need_ij = (bj == 0) || (bi >= 1);
    const bool need_ji = (bi == 0) || (bi == bj);
    double sb = 0.0, tij = 0.0, tji = 0.0;
    for (int c = lane; c < nparts; c += 32) {
        const double* P = part + (int64_t)c * 2 * q2;
        sb += P[q2 + i + (int64_t)q * j];
        if (need_ij) tij += P[i + (int64_t)q * j];
        if (need_ji) tji += P[j + (int64_t)q * i];
    }
    sb = warp_sum(sb);
    tij = warp_sum(tij);
    tji = warp_sum(tji);
    if (lane) return;
    double a;
    if (bi == 0 && bj == 0) a = 0.5 * (sb * (lam[i] + lam[j]) + tij + tji);
    else if (bi == 0) a = lam[i] * sb + tji;           // (AX)^T s_j = lambda_i x_i^T s_j + r_i^T s_j
    else if (bi == bj) a = 0.5 * (tij + tji);
    else a = tij;
    gA[i + (int64_t)q * j] = a;
    gA[j + (int64_t)q * i] = a;
    gB[i + (int64_t)q * j] = sb;
    gB[j + (int64_t)q * i] = sb;
}

// One warp per unordered pair (i <= j): fixed-order sums of the partials.  gramA(i, j) is the
// symmetrised sum inside a diagonal block and the upper-block entry S_i^T AS_j otherwise.
__global__ void k_gram_finalize(int q, int nparts, const double* __restrict__ part, int with_a,
                                double* __restrict__ gA, double* __restrict__ gB,
                                const double* __restrict__ paper_lam, Blocks3 W) {
    const int64_t pair = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t npairs = (int64_t)q * (q + 1) / 2;
    if (pair >= npairs) return;
    int j = 0;
    int64_t u = pair;
    while (u >= j + 1) { u -= j + 1; ++j; }       // column j, row i <= j
    const int i = (int)u;
    const bool same = block_of(W, i) == block_of(W, j);
    const int64_t q2 = (int64_t)q * q;
    double sb = 0.0, sa1 = 0.0, sa2 = 0.0;
    for (int c = lane; c < nparts; c += 32) {
        const double* P = part + (int64_t)c * 2 * q2;
        sb += P[q2 + i + (int64_t)q * j];
        if (with_a) {
            sa1 += P[i + (int64_t)q * j];
            if (same) sa2 += P[j + (int64_t)q * i];
        }
    }
    sb = warp_sum(sb);
    sa1 = warp_sum(sa1);
    sa2 = warp_sum(sa2);
    if (lane) return;
    double a = same ? 0.5 * (sa1 + sa2) : sa1;
    double b = sb;
    if (paper_lam) {
        if (block_of(W, i) == 0 && block_of(W, j) == 0) a = (i == j) ? paper_lam[i] : 0.0;
        if (same) b = (i == j) ? 1.0 : 0.0;
    }
    if (with_a) { gA[i + (int64_t)q * j] = a; gA[j + (int64_t)q * i] = a; }
    gB[i + (int64_t)q * j] = b;
    gB[j + (int64_t)q * i] = b;
}

// ------------------------------------------------------------------ Ritz update

// Pout = S1 C1 + S2 C2 (arithmetic CW, stored TW) and Xout = S0 C0 + Pout (float64).
// S0 is float64; S1, S2 have type TW.  Each thread owns one grid point and kCG output columns.
// CG (float64 blocks only): the coefficients are read from C itself (wide bases whose q x m copy
// would not fit in shared memory); all lanes of a warp read the same entry.
template <typename TW, typename CW, bool CG>
__global__ void k_update(int64_t n, int m, Blocks3 S, const double* __restrict__ C,
                         double* Xout, TW* Pout, float* Xh, float* Xl, int64_t ldout,
                         const unsigned* __restrict__ status, unsigned skip) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int q = S.q();
    if (status && (*status & skip)) return;
    double* cc = reinterpret_cast<double*>(sm_raw);                  // q x m, column-major
    CW* cw = reinterpret_cast<CW*>(sm_raw + sizeof(double) * q * m);  // copy in CW
    if constexpr (!CG) {
        for (int e = threadIdx.y * 32 + threadIdx.x; e < q * m; e += 32 * blockDim.y) {
            cc[e] = C[e];
            cw[e] = (CW)C[e];
        }
    }
    const double* sC = CG ? C : cc;
    const CW* sCw = CG ? reinterpret_cast<const CW*>(C) : cw;
    __syncthreads();
    const int c0 = threadIdx.y * kCG;
    const int w0 = S.w[0], w1 = S.w[1], w2 = S.w[2];
    const int64_t ld = S.ld;
    const double* S0 = static_cast<const double*>(S.p[0]);
    const TW* S1 = static_cast<const TW*>(S.p[1]);
    const TW* S2 = static_cast<const TW*>(S.p[2]);
    for (int64_t base = blockIdx.x * 32ll; base < n; base += (int64_t)gridDim.x * 32) {
        const int64_t p = base + threadIdx.x;
        const bool valid = p < n;
        CW accP[kCG];
        double accX[kCG];
#pragma unroll
        for (int c = 0; c < kCG; ++c) { accP[c] = CW(0); accX[c] = 0.0; }
        if (valid) {
#pragma unroll 8
            for (int i = 0; i < w1; ++i) {
                const CW v = (CW)ld_as(S1 + (int64_t)i * ld + p);
#pragma unroll
                for (int c = 0; c < kCG; ++c) accP[c] = fma(v, sCw[(w0 + i) + q * min(c0 + c, m - 1)], accP[c]);
            }
#pragma unroll 8
            for (int i = 0; i < w2; ++i) {
                const CW v = (CW)ld_as(S2 + (int64_t)i * ld + p);
#pragma unroll
                for (int c = 0; c < kCG; ++c)
                    accP[c] = fma(v, sCw[(w0 + w1 + i) + q * min(c0 + c, m - 1)], accP[c]);
            }
#pragma unroll 8
            for (int i = 0; i < w0; ++i) {
                const double v = __ldg(S0 + (int64_t)i * ld + p);
#pragma unroll
                for (int c = 0; c < kCG; ++c) accX[c] = fma(v, sC[i + q * min(c0 + c, m - 1)], accX[c]);
            }
        }
        __syncthreads();   // every input row of this tile is read before any output is written
        if (valid) {
#pragma unroll
            for (int c = 0; c < kCG; ++c) {
                if (c0 + c < m) {
                    if (Pout) st_as(Pout + (int64_t)(c0 + c) * ldout + p, accP[c]);
                    const double xn = accX[c] + (double)accP[c];
                    Xout[(int64_t)(c0 + c) * ldout + p] = xn;
                    if (Xh) {   // float32 hi / lo planes of X (mixed form)
                        const float hi = (float)xn;
                        Xh[(int64_t)(c0 + c) * ldout + p] = hi;
                        Xl[(int64_t)(c0 + c) * ldout + p] = (float)(xn - (double)hi);
                    }
                }
            }
        }
    }
}

// V <- V Rinv with Rinv upper triangular (b x b, column-major): each thread owns one grid point
// and kCG output columns c0..c0+kCG-1, so it needs input columns 0..c0+kCG-1 only.
// RG (float64 only): Rinv is read from global memory (wide blocks).
template <typename T, bool RG>
__global__ void k_apply_upper(int64_t n, int b, const T* Vin, int64_t ldin, T* Vout, int64_t ldout,
                              const double* __restrict__ Rinv, const unsigned* __restrict__ status,
                              unsigned skip) {
    using C = typename Acc<T>::type;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    if (status && (*status & skip)) return;
    C* r = reinterpret_cast<C*>(sm_raw);
    if constexpr (!RG)
        for (int e = threadIdx.y * 32 + threadIdx.x; e < b * b; e += 32 * blockDim.y) r[e] = (C)Rinv[e];
    const C* sR = RG ? reinterpret_cast<const C*>(Rinv) : r;
    __syncthreads();
    const int c0 = threadIdx.y * kCG;
    const int iend = min(b, c0 + kCG);
    for (int64_t base = blockIdx.x * 32ll; base < n; base += (int64_t)gridDim.x * 32) {
        const int64_t p = base + threadIdx.x;
        const bool valid = p < n;
        C acc[kCG];
#pragma unroll
        for (int c = 0; c < kCG; ++c) acc[c] = C(0);
        if (valid) {
#pragma unroll 8
            for (int i = 0; i < iend; ++i) {
                const C v = (C)Vin[(int64_t)i * ldin + p];
#pragma unroll
                for (int c = 0; c < kCG; ++c) acc[c] = fma(v, sR[i + b * min(c0 + c, b - 1)], acc[c]);
            }
        }
        __syncthreads();   // in place: all inputs of this tile are read before any write
        if (valid) {
#pragma unroll
            for (int c = 0; c < kCG; ++c)
                if (c0 + c < b) Vout[(int64_t)(c0 + c) * ldout + p] = (T)acc[c];
        }
    }
}

}  // namespace

// ====================================================================== launchers
void launch_random_block(uint64_t seed, int64_t n, int m, double* X, int64_t ldx, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(ceil_div(n * m, 256), (int64_t)kNumSMs * 16);
    k_random_block<<<(unsigned)blocks, 256, 0, st>>>(seed, n, m, X, ldx);
    LG_CHECK_LAUNCH();
}

int residual_chunks(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 8 * kResThreads), 2 * kNumSMs));
}

void launch_residual(int64_t n, const ColList& cols, const double* X, const double* AX, int64_t ld,
                     const double* lambda, DType tw, void* W, int64_t ldw, double* partial,
                     cudaStream_t st) {
    if (cols.n <= 0) return;
    const int nchunks = residual_chunks(n);
    const int64_t rows = ceil_div(n, nchunks);
    dim3 grid((unsigned)nchunks, (unsigned)cols.n);
    if (tw == DT_F32)
        k_residual<float><<<grid, kResThreads, 0, st>>>(n, rows, cols, X, AX, ld, lambda, (float*)W, ldw,
                                                        partial, nchunks);
    else
        k_residual<double><<<grid, kResThreads, 0, st>>>(n, rows, cols, X, AX, ld, lambda, (double*)W, ldw,
                                                         partial, nchunks);
    LG_CHECK_LAUNCH();
}

void launch_norms_finalize(int ncols, int nchunks, const double* partial, double* norms,
                           cudaStream_t st) {
    if (ncols <= 0) return;
    k_norms_finalize<<<ncols, 32, 0, st>>>(nchunks, partial, norms);
    LG_CHECK_LAUNCH();
}

// Row ranges of the Gram partial sums: about 1024 rows each, at most 4 per SM, and for wide
// bases at most as many as keep the partial sums (2 q^2 doubles per range) near 256 MB.
int gram_parts(int64_t n, int q) {
    const int64_t cap = std::max<int64_t>(kNumSMs, ((int64_t)1 << 25) / (2 * (int64_t)q * q));
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(ceil_div(n, 1024), 4 * kNumSMs), cap));
}

int64_t gram_scratch_doubles(int64_t n, int q) { return (int64_t)gram_parts(n, q) * 2 * q * q; }

template <typename T0, typename T12, typename C>
static void gram_t(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int nparts,
                   cudaStream_t st) {
    const int q = S.q();
    LG_REQUIRE(q <= kMaxQ, LOBPCG_ERR_ARG, "Gram basis too wide");
    const GramShape gs = gram_shape(S, AS != nullptr, (int)sizeof(C));
    const int threads = (int)ceil_div((int64_t)gs.tpb * gs.ks, 32) * 32;
    LG_REQUIRE(threads <= kGramMaxThreads, LOBPCG_ERR_ARG, "Gram basis too wide");
    const size_t smem = gram_smem_bytes(gs, q, AS != nullptr, (int)sizeof(C));
    LG_REQUIRE(smem <= (size_t)kGramSmemMax, LOBPCG_ERR_ARG, "Gram shared memory too large");
    if (smem > 48 * 1024) {
        static bool attr[64] = {};
        int dev = 0;
        LG_CUDA(cudaGetDevice(&dev));
        if (dev < 64 && !attr[dev]) {
            LG_CUDA(cudaFuncSetAttribute((const void*)k_gram<T0, T12, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kGramSmemMax));
            attr[dev] = true;
        }
    }
    const int64_t rows = ceil_div(n, nparts);
    Blocks3 A = AS ? *AS : S;
    k_gram<T0, T12, C><<<dim3((unsigned)nparts, (unsigned)gs.ngroups), threads, smem, st>>>(n, rows, S, A,
                                                                                           AS ? 1 : 0, part);
}

void launch_gram(int64_t n, const Blocks3& S, const Blocks3* AS, double* part, int nparts,
                 cudaStream_t st) {
    const bool has12 = S.w[1] + S.w[2] > 0;
    const DType t12 = has12 ? S.t12 : S.t0;
    if (S.t0 == DT_F64 && t12 == DT_F64) gram_t<double, double, double>(n, S, AS, part, nparts, st);
    else if (S.t0 == DT_F32 && t12 == DT_F32) gram_t<float, float, float>(n, S, AS, part, nparts, st);
    else throw Error(LOBPCG_ERR_ARG, "unsupported Gram block types");
    LG_CHECK_LAUNCH();
}

void launch_gram_finalize(int q, int nparts, const double* part, bool with_a, double* gramA,
                          double* gramB, const double* paper_lambda, const Blocks3* widths,
                          cudaStream_t st) {
    const int64_t npairs = (int64_t)q * (q + 1) / 2;
    const int64_t threads = npairs * 32;
    Blocks3 W{};
    if (widths) W = *widths;
    else { W.w[0] = q; W.w[1] = 0; W.w[2] = 0; }
    k_gram_finalize<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(
        q, nparts, part, with_a ? 1 : 0, gramA, gramB, paper_lambda, W);
    LG_CHECK_LAUNCH();
}

void launch_apply_rinv(int64_t n, int b, DType t, void* Vin, int64_t ldin, void* Vout,
                       int64_t ldout, const double* Rinv, const unsigned* status,
                       unsigned skip_mask, cudaStream_t st) {
    if (b <= 0) return;
    const int groups = (int)ceil_div(b, kCG);
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 32), (int64_t)kNumSMs * 16);
    if (t == DT_F32) {
        LG_REQUIRE((size_t)b * b * sizeof(float) <= 48 * 1024, LOBPCG_ERR_ARG, "float32 block too wide");
        k_apply_upper<float, false><<<(unsigned)blocks, dim3(32, groups), (size_t)b * b * sizeof(float), st>>>(
            n, b, (const float*)Vin, ldin, (float*)Vout, ldout, Rinv, status, skip_mask);
    } else if ((size_t)b * b * sizeof(double) > 48 * 1024) {
        k_apply_upper<double, true><<<(unsigned)blocks, dim3(32, groups), 0, st>>>(
            n, b, (const double*)Vin, ldin, (double*)Vout, ldout, Rinv, status, skip_mask);
    } else {
        k_apply_upper<double, false><<<(unsigned)blocks, dim3(32, groups), (size_t)b * b * sizeof(double), st>>>(
            n, b, (const double*)Vin, ldin, (double*)Vout, ldout, Rinv, status, skip_mask);
    }
    LG_CHECK_LAUNCH();
}

void launch_update(int64_t n, int m, const Blocks3& S, const double* C, double* Xout, void* Pout,
                   int64_t ldout, const unsigned* status, unsigned skip_mask, cudaStream_t st,
                   float* Xh, float* Xl) {
    const int groups = (int)ceil_div(m, kCG);
    const int64_t blocks = std::min<int64_t>(ceil_div(n, 32), (int64_t)kNumSMs * 16);
    const bool f32 = (S.w[1] + S.w[2] > 0 ? S.t12 : DT_F64) == DT_F32;
    if (f32) {
        const size_t smem = (size_t)S.q() * m * (sizeof(double) + sizeof(float));
        LG_REQUIRE(smem <= 48 * 1024, LOBPCG_ERR_ARG, "float32 update too wide");
        k_update<float, float, false><<<(unsigned)blocks, dim3(32, groups), smem, st>>>(
            n, m, S, C, Xout, (float*)Pout, Xh, Xl, ldout, status, skip_mask);
    } else {
        const size_t smem = (size_t)S.q() * m * (2 * sizeof(double));
        if (smem > 48 * 1024)
            k_update<double, double, true><<<(unsigned)blocks, dim3(32, groups), 0, st>>>(
                n, m, S, C, Xout, (double*)Pout, Xh, Xl, ldout, status, skip_mask);
        else
            k_update<double, double, false><<<(unsigned)blocks, dim3(32, groups), smem, st>>>(
                n, m, S, C, Xout, (double*)Pout, Xh, Xl, ldout, status, skip_mask);
    }
    LG_CHECK_LAUNCH();
}

}  // namespace lg

namespace lg {
void launch_gram_finalize_mx(int q, int m, int b, int bp, int nparts, const double* part,
                             const double* lam, double* gramA, double* gramB, cudaStream_t st) {
    Blocks3 W{};
    W.w[0] = m;
    W.w[1] = b;
    W.w[2] = bp;
    const int64_t wthreads = (int64_t)q * (q + 1) / 2 * 32;
    k_gram_finalize_mx<<<(unsigned)ceil_div(wthreads, 256), 256, 0, st>>>(q, nparts, part, gramA, gramB, lam, W);
    LG_CHECK_LAUNCH();
}
}  // namespace lg

namespace lg {
namespace {
// C (q x b, column-major, q = b + k): rows 0..b-1 the identity, rows b..q-1 minus the cross block
// Y^T V of the Gram matrix G of [V Y] (q x q), so that [V Y] C = V - Y (Y^T V).
__global__ void k_proj_coef(int b, int k, const double* __restrict__ G, double* __restrict__ C) {
    const int q = b + k;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= q * b) return;
    const int i = e % q, j = e / q;
    C[e] = i < b ? (i == j ? 1.0 : 0.0) : -G[j + (int64_t)q * i];
}
}  // namespace

void launch_proj_coef(int b, int k, const double* G, double* C, cudaStream_t st) {
    const int total = (b + k) * b;
    k_proj_coef<<<(unsigned)ceil_div(total, 128), 128, 0, st>>>(b, k, G, C);
    LG_CHECK_LAUNCH();
}
}  // namespace lg
