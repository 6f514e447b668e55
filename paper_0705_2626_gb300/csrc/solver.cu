// LOBPCG driver and the C ABI declared in include/lobpcg_gb300.h.
//
// One handle = one operator (7-point Laplacian on an nx x ny x nz grid), one preconditioner
// (V-cycle hierarchy or identity) and the workspace of a block of m vectors.  The iteration
// follows Section 2.2 of the BLOPEX paper (the algorithm of Section 2.2) with B = I (6m stored vectors), no
// constraints and the soft locking of Section 2.3.  Every step runs in this library's kernels;
// the host only keeps the active index set J, which needs the b residual norms of each
// iteration (one device-to-host copy per iteration, together with a status word that the small
// dense kernels use to report breakdowns).  Nothing on the iteration path falls back to the CPU.
//
// Two forms.  LOBPCG_FP64: every block and every operation in float64.  LOBPCG_MIXED: X, AX and
// all small matrices in float64; W, AW, P, AP, the V-cycle's finest level in float32 and its
// coarser levels stored in bfloat16; the Gram products in float32 with compensated sums.  When
// every implicit residual passes, a float64 correction sweep (the initial orthonormalisation and Rayleigh-Ritz step applied to the current X
// with a fresh float64 A X) recomputes the Ritz pairs and their residuals; columns that fail
// re-enter the loop.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "gram_out.cuh"

using namespace lg;

namespace lg {
std::atomic<long long> g_kernel_launches{0};
thread_local std::string g_handle_free_error;
thread_local int g_wait_limit = -1;
}  // namespace lg

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};
inline double* f64(const Buf& b) { return static_cast<double*>(b.p); }

constexpr int kMaxFp64Sweeps = 16;
// Mixed form: the loop drops a column at kMixedInnerTol * tol, so that the float64 sweep, which
// re-orthonormalises X and rotates it within clusters of close Ritz values, still finds every
// column below tol instead of pushing the ones that passed with no margin back over it.
constexpr double kMixedInnerTol = 0.5;

}  // namespace

struct lobpcg_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    lobpcg_allocator alloc{};
    bool has_alloc = false;
    int precision = LOBPCG_FP64;
    DType tw = DT_F64;      // W / P family and V-cycle level 0
    DType tl = DT_F64;      // V-cycle levels >= 1
    std::string err;
    bool poisoned = false;

    // operator
    bool has_op = false;
    Grid3 g{0, 0, 0};
    double scale = 1.0;
    // preconditioner
    int pc_kind = LOBPCG_PRECOND_NONE;
    int levels = 1, nu_pre = 2, nu_post = 2;
    double omega = 2.0 / 3.0;
    std::vector<Grid3> lv;
    std::vector<double> lscale;
    Buf coarse_tab;
    // variable-coefficient operator: face coefficients per level, dense inverse of the coarsest
    bool varcoef = false;
    std::vector<Buf> lkap;
    Buf vc_inv;
    // options
    int tol_mode = LOBPCG_TOL_RELATIVE, gram_mode = LOBPCG_GRAM_EXPLICIT, phase_timing = 0;
    int gram_engine = LOBPCG_ENGINE_AUTO;       // float32 Grams of the mixed form
    int inner_pcg = 0;                          // inner PCG iterations of the preconditioning (0: V-cycle directly)
    int wait_limit = -1;                        // poll limit of the TMA stage waits (< 0: default)
    Buf pcg_small;                              // inner PCG scalars: rz, rz', pAp (b each), active flags

    // workspace for a block of wm columns
    int wm = 0;
    int64_t ld = 0;
    Buf X, AX;                                  // float64
    Buf W, AW, P, AP, Pc, APc, E0, T0;          // type tw
    Buf Xh, Xl, R;                              // mixed form: float32 planes of X, residual block
    std::vector<Buf> lr, le, lt;                // type tl
    std::vector<int64_t> lld;
    Buf part;          // Gram / residual partial sums
    Buf small;         // gramA, gramB, C, lam, Rinv, norms, rr work
    unsigned* status = nullptr;
    int* colexp = nullptr;     // largest exponent field of each column of the last tensor-core Gram's [S AS]
    int colexp_q = 0;          // its q (0: no valid record)
    size_t part_doubles = 0;
    double *gramA = nullptr, *gramB = nullptr, *Cm = nullptr, *lam = nullptr, *Rinv = nullptr,
           *norms = nullptr, *rrwork = nullptr, *Gsmall = nullptr;

    // user initial block
    Buf X0;
    int X0_m = 0;

    // constraint block Y (the constraint projections): an orthonormal basis Q of span(Y), float64, and its
    // float32 copy for the mixed form; orthonormalised at the first solve after it is set
    Buf Yq, Yq32;
    int ncon = 0;
    bool con_ready = false;

    // solve state
    int state = 0;      // 0 none, 1 iterating, 2 finished
    int m = 0;
    double tol = 0.0;
    int k = 0;
    bool pending_check = false;
    std::vector<int> J;
    std::vector<double> lam_h, norms_h, resid_h;
    std::vector<int> norm_cols;                 // columns whose norms the last residual pass computed
    bool norms_fp64 = true;                     // mixed form: last norms from the float64 sweep
    std::vector<double> norm_by_col;            // those norms, indexed by column
    int p_dropped = 0;
    int fp64_sweeps = 0;
    int final_checks = 0;                       // float64 form: final checks performed
    double setup_ms = 0.0, solve_ms = 0.0;
    double phase_ms[LOBPCG_NPHASES] = {};
    cudaEvent_t ev[LOBPCG_NPHASES + 3] = {};   // phase marks, solve start / end, end of the residual
    long long launches_at_start = 0;
};

namespace {

// ------------------------------------------------------------------ memory
void* dalloc(lobpcg_t* h, size_t bytes) {
    if (bytes == 0) return nullptr;
    void* p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->stream);
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, h->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (!p) throw Error(LOBPCG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    return p;
}

void dfree(lobpcg_t* h, Buf& b) {
    if (b.p) {
        if (h->has_alloc) h->alloc.free(h->alloc.ctx, b.p, b.bytes, (void*)h->stream);
        else cudaFreeAsync(b.p, h->stream);
    }
    b.p = nullptr;
    b.bytes = 0;
}

void ensure(lobpcg_t* h, Buf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return;
    dfree(h, b);
    b.p = dalloc(h, bytes);
    b.bytes = bytes;
}

int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

void free_workspace(lobpcg_t* h) {
    for (Buf* b : {&h->X, &h->AX, &h->W, &h->AW, &h->P, &h->AP, &h->Pc, &h->APc, &h->E0, &h->T0,
                   &h->Xh, &h->Xl, &h->R, &h->part, &h->small})
        dfree(h, *b);
    for (auto& b : h->lr) dfree(h, b);
    for (auto& b : h->le) dfree(h, b);
    for (auto& b : h->lt) dfree(h, b);
    h->lr.clear();
    h->le.clear();
    h->lt.clear();
    h->wm = 0;
    h->status = nullptr;
    h->colexp = nullptr;
    h->colexp_q = 0;
}

void free_varcoef(lobpcg_t* h) {
    for (auto& b : h->lkap) dfree(h, b);
    h->lkap.clear();
    dfree(h, h->vc_inv);
    h->varcoef = false;
}

// Workspace for blocks of up to wm columns (6m vectors of the algorithm + V-cycle buffers).
void ensure_workspace(lobpcg_t* h, int wm) {
    if (h->wm >= wm && h->X.p) return;
    LG_REQUIRE(h->precision == LOBPCG_FP64 || wm <= LOBPCG_MAX_M_MIXED, LOBPCG_ERR_ARG,
               "block wider than the mixed form's limit of 32 columns");
    free_workspace(h);
    h->state = 0;   // a finished or running solve does not survive a reallocation
    const int64_t n = h->g.n();
    h->ld = round_up(n, 32);
    const size_t blk64 = (size_t)h->ld * wm * sizeof(double);
    const size_t blkw = (size_t)h->ld * wm * dtype_size(h->tw);
    ensure(h, h->X, blk64);
    ensure(h, h->AX, blk64);
    for (Buf* b : {&h->W, &h->AW, &h->P, &h->AP, &h->Pc, &h->APc, &h->E0, &h->T0}) ensure(h, *b, blkw);
    if (h->precision == LOBPCG_MIXED)
        for (Buf* b : {&h->Xh, &h->Xl, &h->R}) ensure(h, *b, (size_t)h->ld * wm * sizeof(float));
    const int L = (int)h->lv.size();
    h->lr.assign(L, Buf{});
    h->le.assign(L, Buf{});
    h->lt.assign(L, Buf{});
    h->lld.assign(L, 0);
    for (int l = 1; l < L; ++l) {
        h->lld[l] = round_up(h->lv[l].n(), 32);
        const size_t bytes = (size_t)h->lld[l] * wm * dtype_size(h->tl);
        ensure(h, h->lr[l], bytes);
        ensure(h, h->le[l], bytes);
        ensure(h, h->lt[l], bytes);
    }
    const int q = 3 * wm;
    // the float32 Gram kernels (mixed form and its kernel-level entry points) serve blocks of at
    // most 32 columns
    const int64_t g32 = wm <= LOBPCG_MAX_M_MIXED ? (int64_t)g32_chunks(n) * 2 * q * q : 0;
    h->part_doubles = (size_t)std::max<int64_t>(
        std::max<int64_t>(gram_scratch_doubles(n, q), g32),
        std::max<int64_t>(residual_chunks(n), resid_mx_blocks(h->g)) * wm);
    ensure(h, h->part, h->part_doubles * sizeof(double));
    const size_t nsmall = 2 * (size_t)q * q + (size_t)q * wm + wm + (size_t)wm * wm + wm +
                          (size_t)rr_work_doubles(q) + (size_t)wm * wm + 8 + (size_t)q + 8;
    ensure(h, h->small, nsmall * sizeof(double));
    double* s = f64(h->small);
    h->gramA = s; s += (size_t)q * q;
    h->gramB = s; s += (size_t)q * q;
    h->Cm = s; s += (size_t)q * wm;
    h->lam = s; s += wm;
    h->Rinv = s; s += (size_t)wm * wm;
    h->norms = s; s += wm;
    h->rrwork = s; s += rr_work_doubles(q);
    h->Gsmall = s; s += (size_t)wm * wm;
    h->status = (unsigned*)s;
    h->colexp = reinterpret_cast<int*>(s + 8);           // 2 q ints
    h->colexp_q = 0;
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    h->wm = wm;
}

void require_op(lobpcg_t* h) {
    LG_REQUIRE(h->has_op, LOBPCG_ERR_STATE, "no operator set (call lobpcg_set_operator first)");
}

ColList identity_cols(int b) {
    ColList c{};
    c.n = b;
    for (int i = 0; i < b; ++i) c.idx[i] = i;
    return c;
}

// ------------------------------------------------------------------ operator and T
void spmv(lobpcg_t* h, int ncols, DType t, const void* x, int64_t ldx, void* y, int64_t ldy) {
    if (h->varcoef) {
        launch_vc_sweep(h->g, 0, ncols, f64(h->lkap[0]), h->scale, 0.0, static_cast<const double*>(x), ldx,
                        nullptr, 0, static_cast<double*>(y), ldy, h->stream);
        return;
    }
    launch_stencil_axpby(h->g, ncols, t, 6.0 * h->scale, -h->scale, x, ldx, 0.0, nullptr, 0, y, ldy,
                         h->stream);
}


void copy_cols(lobpcg_t* h, int ncols, int64_t n, DType t, const void* src, int64_t lds, void* dst,
               int64_t ldd) {
    const size_t es = dtype_size(t);
    LG_CUDA(cudaMemcpy2DAsync(dst, ldd * es, src, lds * es, n * es, ncols, cudaMemcpyDeviceToDevice,
                              h->stream));
}

void* col(const Buf& b, DType t, int64_t ld, int j) {
    return static_cast<char*>(b.p) + (size_t)j * ld * dtype_size(t);
}

// V-cycle of the variable-coefficient operator on level l (float64): the steps of vcycle()
// below with the face-coefficient sweeps; the first two pre-smoothing sweeps are not fused.
void vcycle_vc(lobpcg_t* h, int l, int b, const double* r, int64_t ldr, double* e, int64_t lde, double* tmp,
               int64_t ldt) {
    const Grid3& g = h->lv[l];
    const int L = (int)h->lv.size();
    if (l == L - 1) {
        launch_dense_apply((int)g.n(), b, f64(h->vc_inv), r, ldr, e, lde, h->stream);
        return;
    }
    const double s = h->scale, w = h->omega;
    const double* kap = f64(h->lkap[l]);
    double* cur = e;
    int64_t ldc = lde;
    double* oth = tmp;
    int64_t ldo = ldt;
    launch_vc_sweep(g, 3, b, kap, s, w, nullptr, 0, r, ldr, cur, ldc, h->stream);      // from e = 0
    for (int k = 1; k < h->nu_pre; ++k) {
        launch_vc_sweep(g, 1, b, kap, s, w, cur, ldc, r, ldr, oth, ldo, h->stream);
        std::swap(cur, oth);
        std::swap(ldc, ldo);
    }
    launch_vc_sweep(g, 2, b, kap, s, w, cur, ldc, r, ldr, oth, ldo, h->stream);        // r - A e
    const Grid3& gc = h->lv[l + 1];
    double* rc = f64(h->lr[l + 1]);
    double* ec = f64(h->le[l + 1]);
    const int64_t ldl = h->lld[l + 1];
    launch_restrict(g, gc, b, DT_F64, oth, ldo, DT_F64, rc, ldl, h->stream);
    vcycle_vc(h, l + 1, b, rc, ldl, ec, ldl, f64(h->lt[l + 1]), ldl);
    launch_prolong_add(g, gc, b, DT_F64, ec, ldl, DT_F64, cur, ldc, h->stream);
    for (int k = 0; k < h->nu_post; ++k) {
        launch_vc_sweep(g, 1, b, kap, s, w, cur, ldc, r, ldr, oth, ldo, h->stream);
        std::swap(cur, oth);
        std::swap(ldc, ldo);
    }
    if (cur != e) copy_cols(h, b, g.n(), DT_F64, cur, ldc, e, lde);
}

// V-cycle on level l: e = T_l r for b columns of type t.  tmp is a scratch block of the same shape.
void vcycle(lobpcg_t* h, int l, int b, DType t, const void* r, int64_t ldr, void* e, int64_t lde,
            void* tmp, int64_t ldt) {
    const Grid3& g = h->lv[l];
    const int L = (int)h->lv.size();
    const int64_t n = g.n();
    if (l == L - 1) {
        launch_coarse_solve(g, b, t, f64(h->coarse_tab), r, ldr, e, lde, h->stream);
        return;
    }
    if (n <= kFuseMaxPoints && L - l <= kFuseMaxLevels &&
        vcycle_small_smem(h->lv.data() + l, L - l, t) <= 200 * 1024) {
        // the small levels in one kernel (shared memory)
        launch_vcycle_small(h->lv.data() + l, h->lscale.data() + l, L - l, h->omega, h->nu_pre, h->nu_post,
                            f64(h->coarse_tab), b, t, r, ldr, e, lde, h->stream);
        return;
    }
    const double s = h->lscale[l], w = h->omega, alpha = w / (6.0 * s);
    void* cur = e;
    int64_t ldc = lde;
    void* oth = tmp;
    int64_t ldo = ldt;
    auto swap_bufs = [&]() { std::swap(cur, oth); std::swap(ldc, ldo); };
    // pre-smoothing from e = 0; the first sweep (e = alpha r) folds into the second
    int done = 0;
    if (h->nu_pre >= 2) {
        launch_stencil_axpby(g, b, t, alpha * (2.0 - w), alpha * w / 6.0, r, ldr, 0.0, nullptr, 0, cur,
                             ldc, h->stream);
        done = 2;
    } else {
        launch_stencil_axpby(g, b, t, alpha, 0.0, r, ldr, 0.0, nullptr, 0, cur, ldc, h->stream);
        done = 1;
    }
    for (; done < h->nu_pre; ++done) {
        launch_stencil_axpby(g, b, t, 1.0 - w, w / 6.0, cur, ldc, alpha, r, ldr, oth, ldo, h->stream);
        swap_bufs();
    }
    // residual r - A e, restricted to level l+1
    launch_stencil_axpby(g, b, t, -6.0 * s, s, cur, ldc, 1.0, r, ldr, oth, ldo, h->stream);
    const Grid3& gc = h->lv[l + 1];
    const DType tc = h->tl;
    launch_restrict(g, gc, b, t, oth, ldo, tc, h->lr[l + 1].p, h->lld[l + 1], h->stream);
    vcycle(h, l + 1, b, tc, h->lr[l + 1].p, h->lld[l + 1], h->le[l + 1].p, h->lld[l + 1],
           h->lt[l + 1].p, h->lld[l + 1]);
    launch_prolong_add(g, gc, b, tc, h->le[l + 1].p, h->lld[l + 1], t, cur, ldc, h->stream);
    for (int k = 0; k < h->nu_post; ++k) {
        launch_stencil_axpby(g, b, t, 1.0 - w, w / 6.0, cur, ldc, alpha, r, ldr, oth, ldo, h->stream);
        swap_bufs();
    }
    if (cur != e) copy_cols(h, b, n, t, cur, ldc, e, lde);
}

// e = T r (level 0, type t).  tmp: n-by-b scratch of type t, distinct from r and e.
void precond(lobpcg_t* h, int b, DType t, const void* r, int64_t ldr, void* e, int64_t lde,
             void* tmp, int64_t ldt) {
    if (h->pc_kind == LOBPCG_PRECOND_NONE) {
        copy_cols(h, b, h->g.n(), t, r, ldr, e, lde);
        return;
    }
    if (h->varcoef) {
        vcycle_vc(h, 0, b, static_cast<const double*>(r), ldr, static_cast<double*>(e), lde,
                  static_cast<double*>(tmp), ldt);
        return;
    }
    vcycle(h, 0, b, t, r, ldr, e, lde, tmp, ldt);
}

// The preconditioning with an inner PCG solve (Section 4.2): E = T_k(R) = the k-th iterate (k = inner_pcg) of
// PCG for A E = R from E = 0, preconditioned by the V-cycle, columns independent; float64, all
// blocks with the workspace's leading dimension.  R is overwritten (it becomes the PCG residual);
// Z, P, AP and tmp are scratch blocks of b columns.
void inner_pcg(lobpcg_t* h, int b, double* R, double* E, double* Z, double* P, double* AP, double* tmp) {
    const int64_t n = h->g.n(), ld = h->ld;
    cudaStream_t st = h->stream;
    ensure(h, h->pcg_small, (size_t)LOBPCG_MAX_M * (3 * sizeof(double) + sizeof(int)));
    double* rz = f64(h->pcg_small);
    double* rz_new = rz + LOBPCG_MAX_M;
    double* pap = rz_new + LOBPCG_MAX_M;
    int* act = reinterpret_cast<int*>(pap + LOBPCG_MAX_M);
    double* part = f64(h->part);
    LG_REQUIRE((size_t)pcg_chunks(n) * b <= h->part_doubles, LOBPCG_ERR_ARG, "PCG scratch too small");
    LG_CUDA(cudaMemsetAsync(E, 0, (size_t)ld * b * sizeof(double), st));
    precond(h, b, DT_F64, R, ld, Z, ld, tmp, ld);                    // z_0 = M r_0
    copy_cols(h, b, n, DT_F64, Z, ld, P, ld);                        // p_0 = z_0
    launch_fill_int(b, 1, act, st);
    launch_coldot(n, b, R, Z, ld, part, rz, act, st);
    for (int it = 0; it < h->inner_pcg; ++it) {
        spmv(h, b, DT_F64, P, ld, AP, ld);
        launch_coldot(n, b, P, AP, ld, part, pap, act, st);
        launch_pcg_er(n, b, rz, pap, act, E, R, P, AP, ld, st);
        precond(h, b, DT_F64, R, ld, Z, ld, tmp, ld);
        launch_coldot(n, b, R, Z, ld, part, rz_new, act, st);
        launch_pcg_p(n, b, rz_new, rz, act, P, Z, ld, st);
        std::swap(rz, rz_new);
    }
}

// ------------------------------------------------------------------ Gram helpers
Blocks3 blocks(const void* p0, int w0, DType t0, const void* p1, int w1, const void* p2, int w2,
               DType t12, int64_t ld) {
    Blocks3 b{};
    b.p[0] = p0; b.w[0] = w0;
    b.p[1] = w1 ? p1 : p0; b.w[1] = w1;
    b.p[2] = w2 ? p2 : p0; b.w[2] = w2;
    b.ld = ld;
    b.t0 = t0;
    b.t12 = t12;
    return b;
}

// Float64 Gram on the tensor cores (error-free digit products) unless the SIMT engine is chosen
// or the basis is wider than 48 columns.
bool use_oz(const lobpcg_t* h, const Blocks3& S) {
    const bool f64 = S.t0 == DT_F64 && (S.w[1] + S.w[2] == 0 || S.t12 == DT_F64);
    return f64 && h->gram_engine != LOBPCG_ENGINE_SIMT && gram_oz_fits(S.q());
}

// Float64 Y = S C for a tall block S and a small C on the tensor cores (error-free digit products)
// unless the SIMT engine is chosen or the shape is outside the kernel's limits; false if the
// caller must run the float64 FMA kernel instead.
bool tsmm_f64(lobpcg_t* h, const Blocks3& S, const double* C, int ldc, int nx, int np, int w0p, double* out0,
              double* out1, unsigned skip, int scale_mode, const int* sexp) {
    return h->gram_engine != LOBPCG_ENGINE_SIMT &&
           launch_tsmm_oz(h->g.n(), S, C, ldc, nx, np, w0p, out0, out1, S.ld, h->status, skip, h->stream, scale_mode,
                          sexp);
}

// Float64 Ritz update (the Ritz update): Pout = S_1 C_1 + S_2 C_2 (rows >= w0 of C = h->Cm) if Pout is
// not null, and Xout = S C (outputs with the leading dimension of S); in place over S_0 / S_2
// allowed.  side: 0 for S = [X W P], 1 for [AX AW AP]; when the last Gram (the Gram matrices of the Rayleigh-Ritz basis) ran on the
// tensor cores over this basis, its column exponents equilibrate the columns (AX, AW and AP may
// differ in scale by orders of magnitude).
void update_f64(lobpcg_t* h, int m, const Blocks3& S, double* Xout, double* Pout, unsigned skip, int side) {
    const int q = S.q();
    const bool have = h->colexp_q == q;
    if (!tsmm_f64(h, S, h->Cm, q, m, Pout ? m : 0, S.w[0], Xout, Pout, skip, have ? TZ_SCALE_S_COLS : TZ_SCALE_NONE,
                  have ? h->colexp + side * q : nullptr))
        launch_update(h->g.n(), m, S, h->Cm, Xout, Pout, S.ld, h->status, skip, h->stream);
}

// V <- V Rinv (float64, b columns, in place; Rinv b x b upper triangular on the device).  The
// columns of V are equilibrated by the rows of Rinv (R^-1 = D R'^-1 with D the inverse column
// norms), which keeps the product invariant under column scaling of V (Section 2.2).
void apply_rinv_f64(lobpcg_t* h, int b, double* V, const double* Rinv, unsigned skip) {
    const Blocks3 SV = blocks(V, b, DT_F64, nullptr, 0, nullptr, 0, DT_F64, h->ld);
    if (!tsmm_f64(h, SV, Rinv, b, b, 0, 0, V, nullptr, skip, TZ_SCALE_C_ROWS, nullptr))
        launch_apply_rinv(h->g.n(), b, DT_F64, V, h->ld, V, h->ld, Rinv, h->status, skip, h->stream);
}

// Gram matrices of S (and S^T AS).  tensor: the tensor-core digit products may serve (the Grams
// of the Gram matrices of the Rayleigh-Ritz basis); the Cholesky Grams of single blocks pass false and stay on the float64 pipe:
// their factor decides breakdown (R9) and is inverted, and the tensor Grams' errors, relative to
// each window's largest entries, are coarser than those of float64 sums on the nearly dependent
// blocks near convergence (a 128^3, m = 48 solve broke down on W_J with them, converged without).
void gram(lobpcg_t* h, const Blocks3& S, const Blocks3* AS, double* gA, double* gB,
          const double* paper_lam, bool tensor) {
    const int64_t n = h->g.n();
    const int q = S.q();
    h->colexp_q = 0;
    if (tensor && use_oz(h, S)) {
        const int nparts = launch_gram_oz(n, S, AS, f64(h->part), (int64_t)h->part_doubles, h->status, h->stream,
                                          AS ? h->colexp : nullptr);
        if (nparts > 0) {
            if (AS) h->colexp_q = q;
            launch_gram_finalize(q, nparts, f64(h->part), AS != nullptr, gA, gB, paper_lam, &S, h->stream);
            return;
        }
    }
    const int nparts = (int)std::min<int64_t>(gram_parts(n, q), (int64_t)(h->part_doubles / (2 * (size_t)q * q)));
    LG_REQUIRE(nparts >= 1, LOBPCG_ERR_ARG, "Gram scratch too small");
    launch_gram(n, S, AS, f64(h->part), nparts, h->stream);
    launch_gram_finalize(q, nparts, f64(h->part), AS != nullptr, gA, gB, paper_lam, &S, h->stream);
}

int use_tc(const lobpcg_t* h) {
    return h->gram_engine == LOBPCG_ENGINE_TENSOR ? GRAM_TC_ALWAYS
                                                  : (h->gram_engine == LOBPCG_ENGINE_AUTO ? GRAM_TC_WIDE : GRAM_TC_NEVER);
}

// Mixed form: two passes of block Gram-Schmidt of V (b float32 columns) against X (m float64
// columns, its hi plane) and, if W != null, against W (b float32 columns), then the Cholesky
// step of 11 / 15.  The trial subspace of the Rayleigh-Ritz step is unchanged; the basis
// [X W P] becomes well conditioned, which the float32 search directions need (with
// near-dependent columns the float32 roundings of the Gram matrices would be magnified into
// spurious Ritz pairs).
// The second pass computes C2 = [X W]^T V and V^T V of its input; then G = V^T V - C2^T C2 is the
// Gram matrix of V - L C2 (L = [X W] has orthonormal columns to float32 accuracy, and C2 is at
// the float32 rounding level, so the neglected term is ~1e-14), R = chol(G), and one pass writes
// V <- (V - L C2) R^-1 = [L V] [-C2 R^-1; R^-1].  fail_bit: the status bit of a failed Cholesky;
// skip_bits: earlier failures that skip this step.
void project_normalize(lobpcg_t* h, int b, void* V, const void* W, unsigned fail_bit, unsigned skip_bits) {
    const int64_t n = h->g.n();
    const int m = h->m;
    const int wb = W ? b : 0;
    const float* Xh = static_cast<const float*>(h->Xh.p);
    const float* Wf = static_cast<const float*>(W);
    float* Vf = static_cast<float*>(V);
    cudaStream_t st = h->stream;
    // pass 1: V <- V - L (L^T V); the coefficients in gramB, which is free until the Gram matrices of the Rayleigh-Ritz basis
    launch_gram32_cross(n, h->ld, Xh, m, Wf, wb, Vf, b, h->gramB, nullptr, f64(h->part), (int64_t)h->part_doubles,
                        h->status, use_tc(h), st);
    launch_project32(n, b, Vf, Xh, m, Wf, wb, h->ld, h->gramB, m + wb, h->status, st);
    // pass 2: C2 and G, the Cholesky factor, then projection and R^-1 in one pass
    launch_gram32_cross(n, h->ld, Xh, m, Wf, wb, Vf, b, h->gramB, h->Gsmall, f64(h->part), (int64_t)h->part_doubles,
                        h->status, use_tc(h), st);
    launch_gram_sub_ctc(m + wb, b, h->gramB, m + wb, h->Gsmall, st);
    launch_chol_rinv(b, h->Gsmall, h->Rinv, h->status, fail_bit, skip_bits, st);
    const unsigned skip = fail_bit | skip_bits;
    launch_projapply_coef(m + wb, b, h->gramB, m + wb, h->Rinv, h->gramA, h->status, skip, st);
    launch_combine32(n, b, Vf, Xh, m, Wf, wb, h->ld, h->gramA, m + wb + b, h->status, skip, h->status, st);
}

// V <- V Rinv (the orthonormalisations of W and P), in place; skipped on the device if *status & skip.
void apply_rinv(lobpcg_t* h, int b, DType t, void* V, unsigned skip) {
    if (t == DT_F32)
        launch_apply32(h->g.n(), b, static_cast<float*>(V), h->ld, h->Rinv, h->status, skip, h->status, h->stream);
    else
        apply_rinv_f64(h, b, static_cast<double*>(V), h->Rinv, skip);
}

// G = V^T V for the Cholesky orthonormalisation of a W / P block (the orthonormalisations of W and P).
void block_gram(lobpcg_t* h, int b, DType t, const void* V, double* G) {
    if (t == DT_F32) {
        launch_gram32_cross(h->g.n(), h->ld, nullptr, 0, nullptr, 0, static_cast<const float*>(V), b, nullptr, G,
                            f64(h->part), (int64_t)h->part_doubles, h->status, use_tc(h), h->stream);
    } else {
        const Blocks3 S = blocks(V, b, t, nullptr, 0, nullptr, 0, t, h->ld);
        gram(h, S, nullptr, h->gramA, G, nullptr, false);
    }
}

// ------------------------------------------------------------------ timing
struct PhaseTimer {
    lobpcg_t* h;
    bool on;
    explicit PhaseTimer(lobpcg_t* hh) : h(hh), on(hh->phase_timing != 0) {}
    void mark(int i) {
        if (on) LG_CUDA(cudaEventRecord(h->ev[i], h->stream));
    }
};

void events_create(lobpcg_t* h) {
    for (auto& e : h->ev)
        if (!e) LG_CUDA(cudaEventCreate(&e));
}

// ------------------------------------------------------------------ the iteration
void residual_into_W(lobpcg_t* h) {
    h->norms_fp64 = true;
    // the residuals: W[:, t] = AX[:, J[t]] - lambda[J[t]] X[:, J[t]] and the norms (to the host).  The
    // mixed form computes the residual R of all m columns (its Gram uses R for every column).
    const int64_t n = h->g.n();
    const bool mixed = h->precision == LOBPCG_MIXED;
    ColList cols{};
    if (mixed) {
        cols = identity_cols(h->m);
    } else {
        cols.n = (int)h->J.size();
        for (int t = 0; t < cols.n; ++t) cols.idx[t] = h->J[t];
    }
    h->norm_cols.assign(cols.idx, cols.idx + cols.n);
    launch_residual(n, cols, f64(h->X), f64(h->AX), h->ld, h->lam, h->tw, mixed ? h->R.p : h->W.p, h->ld,
                    f64(h->part), h->stream);
    launch_norms_finalize(cols.n, residual_chunks(n), f64(h->part), h->norms, h->stream);
}

// Mixed form, the residuals from the double-float planes of X: R = A X - X Lambda for all m columns.
void residual_from_planes(lobpcg_t* h) {
    const int m = h->m;
    h->norms_fp64 = false;
    h->norm_cols.resize(m);
    for (int j = 0; j < m; ++j) h->norm_cols[j] = j;
    launch_resid_mx(h->g, m, h->scale, static_cast<const float*>(h->Xh.p), static_cast<const float*>(h->Xl.p),
                    h->ld, h->lam, static_cast<float*>(h->R.p), h->ld, f64(h->part), h->stream);
    launch_norms_finalize(m, resid_mx_blocks(h->g), f64(h->part), h->norms, h->stream);
}

// Mixed form: the float64 copy of X (for the float64 sweep and the results) from the planes.
void sync_x_from_planes(lobpcg_t* h) {
    if (h->precision != LOBPCG_MIXED) return;
    launch_planes_to_f64(h->g.n(), h->m, static_cast<const float*>(h->Xh.p), static_cast<const float*>(h->Xl.p),
                         h->ld, f64(h->X), h->ld, h->stream);
}

// Copy the small per-iteration results to the host: norms of J, lambda, status word.
unsigned fetch_small(lobpcg_t* h) {
    unsigned st = 0;
    h->norms_h.resize(h->norm_cols.size());
    if (!h->norm_cols.empty())
        LG_CUDA(cudaMemcpyAsync(h->norms_h.data(), h->norms, h->norm_cols.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, h->stream));
    h->lam_h.resize(h->m);
    LG_CUDA(cudaMemcpyAsync(h->lam_h.data(), h->lam, h->m * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LG_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    LG_CUDA(cudaStreamSynchronize(h->stream));
    h->norm_by_col.assign(h->m, 0.0);
    for (size_t t = 0; t < h->norm_cols.size(); ++t) h->norm_by_col[h->norm_cols[t]] = h->norms_h[t];
    return st;
}

// The initial orthonormalisation and Rayleigh-Ritz step on the current X, all in float64: X = X R^-1 with R = chol(X^T X), AX = A X,
// (X^T AX) TMP = TMP Lambda, X = X TMP, AX = AX TMP; then the residuals for all m columns.
// This is the setup of the algorithm and, in the mixed form, the float64 correction sweep.
// ------------------------------------------------------------------ constraints (the constraint projections)
// The handle keeps an orthonormal basis Q of span(Y); with it the projector
// Y (Y^T Y)^-1 Y^T of the constraint projections (B = I) is Q Q^T, applied chunk by chunk (chunks of Q sized
// so that [V Q_c] fits the Gram scratch of the workspace: b + k <= 3 wm).
void free_constraints(lobpcg_t* h) {
    dfree(h, h->Yq);
    dfree(h, h->Yq32);
    h->ncon = 0;
    h->con_ready = false;
}

// V <- V - Qc (Qc^T V) for one chunk Qc (k columns) of the float64 basis; V float64, b columns.
void project_chunk64(lobpcg_t* h, int b, double* V, const double* Qc, int k) {
    const Blocks3 S = blocks(V, b, DT_F64, Qc, k, nullptr, 0, DT_F64, h->ld);
    gram(h, S, nullptr, h->gramA, h->gramB, nullptr, false);     // gramB = [V Qc]^T [V Qc]
    launch_proj_coef(b, k, h->gramB, h->gramA, h->stream);       // gramA <- [I; -Qc^T V]
    launch_update(h->g.n(), b, S, h->gramA, V, nullptr, h->ld, nullptr, 0u, h->stream);
}

// The constraint projections: V <- V - Y (Y^T Y)^-1 Y^T V for the b columns of V (type t).  Float64: one pass
// over the chunks of Q.  Float32 (mixed form, the constraint projection of W on W_J): two passes of block Gram-Schmidt
// against the float32 copy of Q (the float32 roundings of one pass leave ~1e-7 of span(Y)).
void apply_constraints(lobpcg_t* h, int b, DType t, void* V) {
    if (h->ncon == 0 || b == 0) return;
    const int64_t n = h->g.n();
    const int kc = std::min(32, 2 * h->wm);
    if (t == DT_F64) {
        for (int c0 = 0; c0 < h->ncon; c0 += kc)
            project_chunk64(h, b, static_cast<double*>(V), static_cast<const double*>(col(h->Yq, DT_F64, h->ld, c0)),
                            std::min(kc, h->ncon - c0));
        return;
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int c0 = 0; c0 < h->ncon; c0 += kc) {
            const int k = std::min(kc, h->ncon - c0);
            const float* Qc = static_cast<const float*>(col(h->Yq32, DT_F32, h->ld, c0));
            launch_gram32_cross(n, h->ld, Qc, k, nullptr, 0, static_cast<const float*>(V), b, h->gramB, nullptr,
                                f64(h->part), (int64_t)h->part_doubles, h->status, use_tc(h), h->stream);
            launch_project32(n, b, static_cast<float*>(V), Qc, k, nullptr, 0, h->ld, h->gramB, k, h->status,
                             h->stream);
        }
}

// Orthonormalise the constraint block in place (block Gram-Schmidt against the earlier chunks and
// Cholesky QR within a chunk, each twice), then the float32 copy.  ERR_BREAKDOWN if Y^T Y is not
// numerically positive definite.
void prepare_constraints(lobpcg_t* h) {
    if (h->ncon == 0 || h->con_ready) return;
    const int64_t n = h->g.n();
    cudaStream_t st = h->stream;
    const int kc = std::max(1, std::min(32, (3 * h->wm) / 2));
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
    for (int c0 = 0; c0 < h->ncon; c0 += kc) {
        const int k = std::min(kc, h->ncon - c0);
        double* Yk = static_cast<double*>(col(h->Yq, DT_F64, h->ld, c0));
        for (int pass = 0; pass < 2; ++pass) {
            for (int j0 = 0; j0 < c0; j0 += kc)
                project_chunk64(h, k, Yk, static_cast<const double*>(col(h->Yq, DT_F64, h->ld, j0)),
                                std::min(kc, c0 - j0));
            const Blocks3 S = blocks(Yk, k, DT_F64, nullptr, 0, nullptr, 0, DT_F64, h->ld);
            gram(h, S, nullptr, h->gramA, h->gramB, nullptr, false);
            launch_chol_rinv(k, h->gramB, h->gramA, h->status, ST_X_BREAKDOWN, 0u, st);
            apply_rinv_f64(h, k, Yk, h->gramA, ST_X_BREAKDOWN);
        }
    }
    unsigned stw = 0;
    LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    LG_CUDA(cudaStreamSynchronize(st));
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
    if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    if (stw & (ST_X_BREAKDOWN | ST_NONFINITE))
        throw Error(LOBPCG_ERR_BREAKDOWN, "the constraint block Y is not numerically linearly independent");
    if (h->precision == LOBPCG_MIXED) {
        ensure(h, h->Yq32, (size_t)h->ld * h->ncon * sizeof(float));
        launch_convert(n, h->ncon, DT_F64, h->Yq.p, h->ld, DT_F32, h->Yq32.p, h->ld, st);
    }
    h->con_ready = true;
}

void orthonormalize_and_rr(lobpcg_t* h) {
    const int64_t n = h->g.n();
    const int m = h->m;
    cudaStream_t st = h->stream;
    const Blocks3 SX = blocks(h->X.p, m, DT_F64, nullptr, 0, nullptr, 0, DT_F64, h->ld);
    gram(h, SX, nullptr, h->gramA, h->Gsmall, nullptr, false);
    launch_chol_rinv(m, h->Gsmall, h->Rinv, h->status, ST_X_BREAKDOWN, 0u, st);
    apply_rinv_f64(h, m, f64(h->X), h->Rinv, ST_X_BREAKDOWN);
    spmv(h, m, DT_F64, h->X.p, h->ld, h->AX.p, h->ld);
    const Blocks3 SAX = blocks(h->AX.p, m, DT_F64, nullptr, 0, nullptr, 0, DT_F64, h->ld);
    gram(h, SX, &SAX, h->gramA, h->gramB, nullptr, true);
    launch_rayleigh_ritz(m, m, m, h->gramA, nullptr, h->lam, h->Cm, h->rrwork, h->status,
                         ST_X_BREAKDOWN, st);
    const unsigned skip = ST_X_BREAKDOWN | ST_RR_BREAKDOWN;
    float* xh = h->precision == LOBPCG_MIXED ? static_cast<float*>(h->Xh.p) : nullptr;
    float* xl = h->precision == LOBPCG_MIXED ? static_cast<float*>(h->Xl.p) : nullptr;
    if (xh) launch_update(n, m, SX, h->Cm, f64(h->X), nullptr, h->ld, h->status, skip, st, xh, xl);
    else update_f64(h, m, SX, f64(h->X), nullptr, skip, 0);
    update_f64(h, m, SAX, f64(h->AX), nullptr, skip, 1);
    h->J.resize(m);
    for (int j = 0; j < m; ++j) h->J[j] = j;
    residual_into_W(h);
}

void check_setup_status(lobpcg_t* h, unsigned stw) {
    if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    if (stw & ST_NONFINITE) throw Error(LOBPCG_ERR_NONFINITE, "non-finite entry in the block X");
    if (stw & (ST_X_BREAKDOWN | ST_RR_BREAKDOWN))
        throw Error(LOBPCG_ERR_BREAKDOWN, "X^T X is not numerically positive definite (the orthonormalisation of X)");
    for (double v : h->lam_h)
        if (!std::isfinite(v)) throw Error(LOBPCG_ERR_NONFINITE, "non-finite Ritz value");
}

void begin(lobpcg_t* h, int m, double tol, uint64_t seed) {
    require_op(h);
    const int64_t n = h->g.n();
    LG_REQUIRE(m >= 1 && m <= LOBPCG_MAX_M, LOBPCG_ERR_ARG, "m out of range [1, 100]");
    LG_REQUIRE(h->precision == LOBPCG_FP64 || m <= LOBPCG_MAX_M_MIXED, LOBPCG_ERR_ARG,
               "m out of range [1, 32] for the mixed form");
    LG_REQUIRE(2 * (int64_t)m <= n, LOBPCG_ERR_ARG, "m too large for the grid (need m <= n/2)");
    LG_REQUIRE(2 * ((int64_t)m + h->ncon) <= n, LOBPCG_ERR_ARG,
               "m plus the constraint columns too large for the grid (need m + l <= n/2)");
    LG_REQUIRE(tol >= 0.0 && std::isfinite(tol), LOBPCG_ERR_ARG, "tol must be finite and >= 0");
    ensure_workspace(h, m);
    events_create(h);
    h->m = m;
    h->tol = tol;
    h->k = 0;
    h->p_dropped = 0;
    h->fp64_sweeps = 0;
    h->final_checks = 0;
    h->J.clear();
    std::fill(h->phase_ms, h->phase_ms + LOBPCG_NPHASES, 0.0);
    h->state = 0;
    cudaStream_t st = h->stream;
    LG_CUDA(cudaEventRecord(h->ev[LOBPCG_NPHASES], st));
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
    // input block
    if (h->X0.p && h->X0_m == m) copy_cols(h, m, n, DT_F64, h->X0.p, n, h->X.p, h->ld);
    else launch_random_block(seed, n, m, f64(h->X), h->ld, st);
    // the constraint projection of X: apply the constraints to X
    prepare_constraints(h);
    apply_constraints(h, m, DT_F64, h->X.p);
    // the set-up and the residuals of k = 0
    orthonormalize_and_rr(h);
    LG_CUDA(cudaEventRecord(h->ev[LOBPCG_NPHASES + 1], st));
    const unsigned stw = fetch_small(h);
    float ms = 0.f;
    LG_CUDA(cudaEventElapsedTime(&ms, h->ev[LOBPCG_NPHASES], h->ev[LOBPCG_NPHASES + 1]));
    h->setup_ms = ms;
    h->solve_ms = 0.0;
    check_setup_status(h, stw);
    h->pending_check = true;
    h->state = 1;
}

// The residuals and the soft-locking test with the norms of the last residual pass: shrink J.  Returns true if J is empty.
bool check_and_lock(lobpcg_t* h) {
    if (!h->pending_check) return h->J.empty();
    h->pending_check = false;
    for (double v : h->norms_h)
        if (!std::isfinite(v)) throw Error(LOBPCG_ERR_NONFINITE, "non-finite residual norm");
    auto bound_of = [&](int j) {
        double bound = h->tol_mode == LOBPCG_TOL_RELATIVE ? h->tol * std::fabs(h->lam_h[j]) : h->tol;
        if (h->precision == LOBPCG_MIXED && !h->norms_fp64) bound *= kMixedInnerTol;
        return bound;
    };
    if (h->precision == LOBPCG_MIXED) {
        // The mixed form has the residuals of all m columns every pass and re-activates a
        // soft-locked column whose residual grew again: the Rayleigh-Ritz step keeps rotating
        // locked columns, and inside a cluster of equal Ritz values it can move the error of an
        // active column into a locked one.  (The float64 form keeps the paper's rule: J only
        // shrinks.)
        std::vector<int> nJ;
        for (int j = 0; j < h->m; ++j)
            if (!(h->norm_by_col[j] <= bound_of(j))) nJ.push_back(j);
        h->J.swap(nJ);
        return h->J.empty();
    }
    std::vector<int> keep;   // positions t in the old J that stay active
    for (size_t t = 0; t < h->J.size(); ++t) {
        const int j = h->J[t];
        if (!(h->norm_by_col[j] <= bound_of(j))) keep.push_back((int)t);
    }
    if (keep.size() != h->J.size()) {
        // compact the residual block W to the surviving columns
        std::vector<int> nJ;
        const size_t es = dtype_size(h->tw);
        for (size_t u = 0; u < keep.size(); ++u) {
            if ((int)u != keep[u])
                LG_CUDA(cudaMemcpyAsync(col(h->W, h->tw, h->ld, (int)u), col(h->W, h->tw, h->ld, keep[u]),
                                        h->g.n() * es, cudaMemcpyDeviceToDevice, h->stream));
            nJ.push_back(h->J[keep[u]]);
        }
        h->J.swap(nJ);
    }
    return h->J.empty();
}

// The iteration from the preconditioning on for the current J, then the residuals of the next pass.
void pass_body(lobpcg_t* h) {
    const int64_t n = h->g.n();
    const int m = h->m, b = (int)h->J.size();
    const int64_t ld = h->ld;
    const DType tw = h->tw;
    cudaStream_t st = h->stream;
    PhaseTimer tm(h);
    tm.mark(0);
    // the preconditioning: W_J = T W_J (output in E0, then the buffers swap roles).  The mixed form keeps the
    // residuals of all columns in R and preconditions R[:, J].
    const bool mixed = h->precision == LOBPCG_MIXED;
    const void* rin = h->W.p;
    if (mixed) {
        if (b == m) {
            rin = h->R.p;
        } else {
            for (int t = 0; t < b; ++t)
                LG_CUDA(cudaMemcpyAsync(col(h->W, tw, ld, t), col(h->R, tw, ld, h->J[t]), n * dtype_size(tw),
                                        cudaMemcpyDeviceToDevice, st));
        }
    }
    if (h->inner_pcg > 0 && !mixed)
        inner_pcg(h, b, f64(h->W), f64(h->E0), f64(h->Pc), f64(h->APc), f64(h->AW), f64(h->T0));
    else
        precond(h, b, tw, rin, ld, h->E0.p, ld, h->T0.p, ld);
    std::swap(h->W, h->E0);
    tm.mark(1);
    // the constraint projection of W: apply the constraints to the preconditioned residuals
    apply_constraints(h, b, tw, h->W.p);
    // the orthonormalisation of W: W_J = W_J R^-1, R = chol(W_J^T W_J) (the mixed form first projects W_J against X)
    if (mixed) {
        project_normalize(h, b, h->W.p, nullptr, ST_W_BREAKDOWN, 0u);
    } else {
        block_gram(h, b, tw, h->W.p, h->Gsmall);
        launch_chol_rinv(b, h->Gsmall, h->Rinv, h->status, ST_W_BREAKDOWN, 0u, st);
        apply_rinv(h, b, tw, h->W.p, ST_W_BREAKDOWN);
    }
    tm.mark(2);
    // the product A W: AW_J = A W_J
    spmv(h, b, tw, h->W.p, ld, h->AW.p, ld);
    tm.mark(3);
    // the orthonormalisation of P: P_J = P_J R^-1, AP_J = AP_J R^-1 with R = chol(P_J^T P_J)
    const bool use_p = h->k > 0;
    void* Pj = h->P.p;
    void* APj = h->AP.p;
    if (use_p) {
        if (b != m) {
            const size_t es = dtype_size(tw);
            for (int t = 0; t < b; ++t) {
                LG_CUDA(cudaMemcpyAsync(col(h->Pc, tw, ld, t), col(h->P, tw, ld, h->J[t]), n * es,
                                        cudaMemcpyDeviceToDevice, st));
                if (h->precision != LOBPCG_MIXED)
                    LG_CUDA(cudaMemcpyAsync(col(h->APc, tw, ld, t), col(h->AP, tw, ld, h->J[t]), n * es,
                                            cudaMemcpyDeviceToDevice, st));
            }
            Pj = h->Pc.p;
            APj = h->APc.p;
        }
        if (mixed) {
            project_normalize(h, b, Pj, h->W.p, ST_P_DROPPED, ST_W_BREAKDOWN);
        } else {
            block_gram(h, b, tw, Pj, h->Gsmall);
            launch_chol_rinv(b, h->Gsmall, h->Rinv, h->status, ST_P_DROPPED, ST_W_BREAKDOWN, st);
            apply_rinv(h, b, tw, Pj, ST_W_BREAKDOWN | ST_P_DROPPED);
        }
        if (h->precision == LOBPCG_MIXED) {
            // Mixed form: AP_J = A P_J by one more (float32) SpMV.  P_J is nearly rank deficient
            // near convergence, and R^-1 would magnify the separate float32 roundings of P_J and
            // AP_J so much that AP_J R^-1 no longer matches A (P_J R^-1).
            spmv(h, b, tw, Pj, ld, APj, ld);
        } else {
            apply_rinv_f64(h, b, static_cast<double*>(APj), h->Rinv, ST_W_BREAKDOWN | ST_P_DROPPED);
        }
    }
    tm.mark(4);
    // the Gram matrices of the Rayleigh-Ritz basis: Gram matrices of the basis [X W_J P_J]
    const Blocks3 S = blocks(h->X.p, m, DT_F64, h->W.p, b, Pj, use_p ? b : 0, tw, ld);
    const Blocks3 AS = blocks(h->AX.p, m, DT_F64, h->AW.p, b, APj, use_p ? b : 0, tw, ld);
    const int q = S.q();
    if (mixed) {
        auto F = [](const void* p) { return static_cast<const float*>(p); };
        launch_gram_mx2(n, ld, F(h->Xh.p), F(h->Xl.p), F(h->W.p), F(Pj), F(h->R.p), F(h->AW.p), F(APj), m, b,
                        use_p ? b : 0, f64(h->part), (int64_t)h->part_doubles, h->lam, h->gramA, h->gramB, h->status,
                        use_tc(h), st);
    } else {
        gram(h, S, &AS, h->gramA, h->gramB, h->gram_mode == LOBPCG_GRAM_PAPER ? h->lam : nullptr, true);
    }
    tm.mark(5);
    // the Rayleigh-Ritz step: gramA C = gramB C Lambda (P block dropped on device if needed)
    launch_rayleigh_ritz(q, m + b, m, h->gramA, h->gramB, h->lam, h->Cm, h->rrwork, h->status,
                         ST_W_BREAKDOWN, st);
    tm.mark(6);
    // the Ritz update: P = W_J C_W + P_J C_P, X = X C_X + P (and the A-side)
    const unsigned skip = ST_W_BREAKDOWN | ST_RR_BREAKDOWN;
    if (mixed) {
        // Mixed form: X as double-float planes; no AX update -- the next residual applies A to X
        // directly (free of the drift that float32 AP would add to an implicitly updated AX),
        // and AP is recomputed from P in the next pass.
        launch_update_mx2(n, m, static_cast<float*>(h->Xh.p), static_cast<float*>(h->Xl.p),
                          static_cast<const float*>(h->W.p), b, static_cast<const float*>(Pj), use_p ? b : 0, ld,
                          h->Cm, q, static_cast<float*>(h->P.p), h->status, skip, h->status, st);
    } else {
        update_f64(h, m, S, f64(h->X), f64(h->P), skip, 0);
        update_f64(h, m, AS, f64(h->AX), f64(h->AP), skip, 1);
    }
    tm.mark(7);
    // the residuals of the next pass
    if (mixed) residual_from_planes(h);
    else residual_into_W(h);
    if (tm.on) LG_CUDA(cudaEventRecord(h->ev[LOBPCG_NPHASES + 2], st));
    const unsigned stw = fetch_small(h);
    if (h->phase_timing) {
        // events 0..7 bracket phases 1..7 of this pass; the residual phase is the tail
        for (int i = 0; i < 7; ++i) {
            float ms = 0.f;
            LG_CUDA(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
            h->phase_ms[i + 1] += ms;
        }
        float ms = 0.f;
        LG_CUDA(cudaEventElapsedTime(&ms, h->ev[7], h->ev[LOBPCG_NPHASES + 2]));
        h->phase_ms[LOBPCG_PH_RESIDUAL] += ms;
    }
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
    if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    if (stw & ST_P_DROPPED) ++h->p_dropped;
    if (stw & ST_W_BREAKDOWN)
        throw Error(LOBPCG_ERR_BREAKDOWN, "W_J^T W_J is not numerically positive definite (the orthonormalisation of W)");
    if (stw & ST_RR_BREAKDOWN)
        throw Error(LOBPCG_ERR_BREAKDOWN, "gramB is not numerically positive definite (the Rayleigh-Ritz step)");
    if (stw & ST_NONFINITE) throw Error(LOBPCG_ERR_NONFINITE, "non-finite Ritz value");
    h->k += 1;
    h->pending_check = true;
}

// Mixed form, once every implicit residual passed: float64 correction sweep on X.  Afterwards J
// holds the columns whose float64 residual still fails.
void fp64_correction(lobpcg_t* h) {
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    sync_x_from_planes(h);
    apply_constraints(h, h->m, DT_F64, h->X.p);     // the constraint projection of X in float64 before the initial orthonormalisation and Rayleigh-Ritz step
    orthonormalize_and_rr(h);
    const unsigned stw = fetch_small(h);
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    check_setup_status(h, stw);
    ++h->fp64_sweeps;
    h->pending_check = true;
}

// Float64 form, once J is empty: the final check.  Soft-locked columns stay in the Rayleigh-Ritz
// basis (Section 2.3) and, inside a cluster of equal Ritz values, the Rayleigh-Ritz rotation can lift a
// locked column above the tolerance after its test.  So A X is recomputed (it replaces the
// implicitly updated AX), the residuals of all m columns are tested, and the failing ones re-enter
// J (check_and_lock compacts W to them).  The solve converges only when this check passes.
void fp64_final_check(lobpcg_t* h) {
    const int m = h->m;
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    spmv(h, m, DT_F64, h->X.p, h->ld, h->AX.p, h->ld);
    h->J.resize(m);
    for (int j = 0; j < m; ++j) h->J[j] = j;
    residual_into_W(h);
    const unsigned stw = fetch_small(h);
    LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
    ++h->final_checks;
    h->pending_check = true;
}

// Residuals of all m columns from A X (not the implicitly updated AX); host resid.
void finish(lobpcg_t* h) {
    const int64_t n = h->g.n();
    const int m = h->m;
    sync_x_from_planes(h);
    spmv(h, m, DT_F64, h->X.p, h->ld, h->AX.p, h->ld);
    ColList cols = identity_cols(m);
    launch_residual(n, cols, f64(h->X), f64(h->AX), h->ld, h->lam, DT_F64, nullptr, 0, f64(h->part),
                    h->stream);
    launch_norms_finalize(m, residual_chunks(n), f64(h->part), h->norms, h->stream);
    h->resid_h.resize(m);
    LG_CUDA(cudaMemcpyAsync(h->resid_h.data(), h->norms, m * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    h->lam_h.resize(m);
    LG_CUDA(cudaMemcpyAsync(h->lam_h.data(), h->lam, m * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
    LG_CUDA(cudaStreamSynchronize(h->stream));
    h->state = 2;
}

void fill_info(lobpcg_t* h, lobpcg_info* out, int status) {
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->status = status;
    out->iters = h->k;
    out->active = (int)h->J.size();
    out->p_dropped = h->p_dropped;
    out->fp64_sweeps = h->precision == LOBPCG_MIXED ? h->fp64_sweeps : h->final_checks;
    double mr = 0.0;
    for (int j = 0; j < (int)h->resid_h.size() && j < (int)h->lam_h.size(); ++j)
        mr = std::max(mr, h->resid_h[j] / std::fabs(h->lam_h[j]));
    out->max_rel_resid = mr;
    out->setup_ms = h->setup_ms;
    out->solve_ms = h->solve_ms;
    out->kernel_launches = g_kernel_launches.load() - h->launches_at_start;
    for (int i = 0; i < LOBPCG_NPHASES; ++i) out->phase_ms[i] = h->phase_ms[i];
}

// Passes until J is empty (in the mixed form: confirmed by the float64 correction sweep) or
// `steps` passes ran.  Returns OK / NOT_CONVERGED.
int run_passes(lobpcg_t* h, int steps) {
    LG_CUDA(cudaEventRecord(h->ev[LOBPCG_NPHASES], h->stream));
    int rc = LOBPCG_NOT_CONVERGED;
    for (int s = 0; s <= steps; ++s) {
        bool empty = check_and_lock(h);
        if (empty && h->precision == LOBPCG_MIXED) {
            if (h->fp64_sweeps >= kMaxFp64Sweeps) break;   // not confirmed: NOT_CONVERGED
            fp64_correction(h);
            empty = check_and_lock(h);
        } else if (empty) {
            fp64_final_check(h);
            empty = check_and_lock(h);
        }
        if (empty) { rc = LOBPCG_OK; break; }
        if (s == steps) break;
        pass_body(h);
    }
    LG_CUDA(cudaEventRecord(h->ev[LOBPCG_NPHASES + 1], h->stream));
    LG_CUDA(cudaEventSynchronize(h->ev[LOBPCG_NPHASES + 1]));
    float ms = 0.f;
    LG_CUDA(cudaEventElapsedTime(&ms, h->ev[LOBPCG_NPHASES], h->ev[LOBPCG_NPHASES + 1]));
    h->solve_ms += ms;
    return rc;
}

// ------------------------------------------------------------------ C-ABI plumbing
// The handle's stage-wait limit for the duration of one call on the calling thread.
struct WaitLimitScope {
    explicit WaitLimitScope(int limit) { g_wait_limit = limit; }
    ~WaitLimitScope() { g_wait_limit = -1; }
};

template <class F>
int guarded(lobpcg_t* h, F&& f) {
    if (!h) return LOBPCG_ERR_ARG;
    if (h->poisoned) return LOBPCG_ERR_CUDA;
    WaitLimitScope wait_scope(h->wait_limit);
    try {
        LG_CUDA(cudaSetDevice(h->device));
        h->err.clear();
        return f();
    } catch (const Error& e) {
        h->err = e.what();
        if (e.code == LOBPCG_ERR_CUDA) h->poisoned = true;
        return e.code;
    } catch (const std::bad_alloc&) {
        h->err = "host allocation failed";
        return LOBPCG_ERR_OOM;
    } catch (const std::exception& e) {
        h->err = e.what();
        return LOBPCG_ERR_ARG;
    }
}

bool valid_ld(int64_t ld, int64_t n) { return ld >= n; }

}  // namespace
// ====================================================================== C ABI
extern "C" {

int lobpcg_create(lobpcg_t** out, int device, void* stream, const lobpcg_allocator* alloc,
                  int precision) {
    if (!out) return LOBPCG_ERR_ARG;
    *out = nullptr;
    if (precision != LOBPCG_FP64 && precision != LOBPCG_MIXED) {
        g_handle_free_error = "precision must be LOBPCG_FP64 or LOBPCG_MIXED";
        return LOBPCG_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_handle_free_error = "invalid CUDA device";
        return device < 0 ? LOBPCG_ERR_ARG : LOBPCG_ERR_CUDA;
    }
    if (alloc && (!alloc->alloc || !alloc->free)) {
        g_handle_free_error = "allocator needs both alloc and free";
        return LOBPCG_ERR_ARG;
    }
    lobpcg_t* h = new (std::nothrow) lobpcg_t();
    if (!h) return LOBPCG_ERR_OOM;
    h->device = device;
    h->stream = (cudaStream_t)stream;
    h->precision = precision;
    h->tw = precision == LOBPCG_MIXED ? DT_F32 : DT_F64;
    h->tl = precision == LOBPCG_MIXED ? DT_BF16 : DT_F64;
    if (alloc) {
        h->alloc = *alloc;
        h->has_alloc = true;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        g_handle_free_error = "cudaSetDevice failed";
        return LOBPCG_ERR_CUDA;
    }
    g_handle_free_error.clear();
    *out = h;
    return LOBPCG_OK;
}

int lobpcg_set_operator(lobpcg_t* h, int kind, int nx, int ny, int nz, double scale,
                        const double* kappa_faces) {
    return guarded(h, [&] {
        LG_REQUIRE(kind == LOBPCG_LAPLACE7 || kind == LOBPCG_VARCOEF7, LOBPCG_ERR_ARG, "unknown operator kind");
        LG_REQUIRE(kind == LOBPCG_VARCOEF7 || kappa_faces == nullptr, LOBPCG_ERR_ARG,
                   "kappa_faces must be NULL for LAPLACE7");
        LG_REQUIRE(kind == LOBPCG_LAPLACE7 || kappa_faces != nullptr, LOBPCG_ERR_ARG,
                   "VARCOEF7 needs kappa_faces");
        LG_REQUIRE(kind == LOBPCG_LAPLACE7 || h->precision == LOBPCG_FP64, LOBPCG_ERR_ARG,
                   "VARCOEF7 needs a LOBPCG_FP64 handle");
        LG_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1, LOBPCG_ERR_ARG, "grid dimensions must be >= 1");
        LG_REQUIRE((int64_t)nx * ny * nz <= (int64_t)1 << 31, LOBPCG_ERR_ARG, "grid too large");
        LG_REQUIRE(scale > 0.0 && std::isfinite(scale), LOBPCG_ERR_ARG, "scale must be > 0");
        free_workspace(h);
        dfree(h, h->coarse_tab);
        dfree(h, h->X0);
        dfree(h, h->pcg_small);
        free_varcoef(h);
        free_constraints(h);
        h->X0_m = 0;
        h->g = Grid3{nx, ny, nz};
        h->scale = scale;
        if (kind == LOBPCG_VARCOEF7) {
            const size_t bytes = (size_t)vc_num_faces(h->g) * sizeof(double);
            h->lkap.assign(1, Buf{});
            ensure(h, h->lkap[0], bytes);
            LG_CUDA(cudaMemcpyAsync(h->lkap[0].p, kappa_faces, bytes, cudaMemcpyDefault, h->stream));
            LG_CUDA(cudaStreamSynchronize(h->stream));
            h->varcoef = true;
        }
        h->has_op = true;
        h->pc_kind = LOBPCG_PRECOND_NONE;
        h->lv.assign(1, h->g);
        h->lscale.assign(1, scale);
        h->state = 0;
        return LOBPCG_OK;
    });
}

int lobpcg_set_preconditioner(lobpcg_t* h, int kind, int levels, int nu_pre, int nu_post,
                              double omega) {
    return guarded(h, [&] {
        require_op(h);
        LG_REQUIRE(kind == LOBPCG_PRECOND_NONE || kind == LOBPCG_PRECOND_GMG, LOBPCG_ERR_ARG,
                   "unknown preconditioner kind");
        free_workspace(h);
        dfree(h, h->coarse_tab);
        for (size_t l = 1; l < h->lkap.size(); ++l) dfree(h, h->lkap[l]);
        if (h->varcoef) h->lkap.resize(1);
        dfree(h, h->vc_inv);
        h->lv.assign(1, h->g);
        h->lscale.assign(1, h->scale);
        h->pc_kind = LOBPCG_PRECOND_NONE;
        if (kind == LOBPCG_PRECOND_NONE) return LOBPCG_OK;
        LG_REQUIRE(levels >= 1 && levels <= 24, LOBPCG_ERR_ARG, "levels out of range");
        LG_REQUIRE(nu_pre >= 1 && nu_post == nu_pre, LOBPCG_ERR_ARG,
                   "need nu_pre == nu_post >= 1 (a symmetric V-cycle)");
        LG_REQUIRE(omega > 0.0 && omega <= 1.0, LOBPCG_ERR_ARG, "omega must be in (0, 1]");
        std::vector<Grid3> lv{h->g};
        std::vector<double> ls{h->scale};
        for (int l = 1; l < levels; ++l) {
            const Grid3 p = lv.back();
            const Grid3 c{p.nx / 2, p.ny / 2, p.nz / 2};
            LG_REQUIRE(c.nx >= 1 && c.ny >= 1 && c.nz >= 1, LOBPCG_ERR_ARG,
                       "grid cannot be coarsened to that many levels");
            lv.push_back(c);
            ls.push_back(ls.back() / 4.0);
        }
        LG_REQUIRE(lv.back().n() <= (h->varcoef ? 512 : 4096), LOBPCG_ERR_ARG,
                   h->varcoef ? "coarsest level has more than 512 points; use more levels"
                              : "coarsest level has more than 4096 points; use more levels");
        h->lv = lv;
        h->lscale = ls;
        h->levels = levels;
        h->nu_pre = nu_pre;
        h->nu_post = nu_post;
        h->omega = omega;
        if (h->varcoef) {
            // coarse face coefficients level by level, then the dense inverse of the coarsest
            h->lkap.resize(1);
            for (int l = 1; l < levels; ++l) {
                h->lkap.push_back(Buf{});
                ensure(h, h->lkap[l], (size_t)vc_num_faces(lv[l]) * sizeof(double));
                launch_vc_coarsen(lv[l - 1], lv[l], f64(h->lkap[l - 1]), f64(h->lkap[l]), h->stream);
            }
            const int64_t nc = lv.back().n();
            ensure(h, h->vc_inv, (size_t)(3 * nc * nc + 2) * sizeof(double));
            double* A = f64(h->vc_inv) + nc * nc;
            int* fail = reinterpret_cast<int*>(f64(h->vc_inv) + 3 * nc * nc);
            LG_CUDA(cudaMemsetAsync(fail, 0, sizeof(int), h->stream));
            launch_vc_coarse_inverse(lv.back(), f64(h->lkap.back()), h->scale, A, A + nc * nc, f64(h->vc_inv), fail,
                                     h->stream);
            int fail_h = 0;
            LG_CUDA(cudaMemcpyAsync(&fail_h, fail, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            LG_CUDA(cudaStreamSynchronize(h->stream));
            LG_REQUIRE(!fail_h, LOBPCG_ERR_ARG, "coarsest operator is not positive definite (kappa must be > 0)");
        } else {
            ensure(h, h->coarse_tab, coarse_tables_size(lv.back()) * sizeof(double));
            launch_coarse_setup(lv.back(), ls.back(), f64(h->coarse_tab), h->stream);
        }
        h->pc_kind = LOBPCG_PRECOND_GMG;
        h->state = 0;
        return LOBPCG_OK;
    });
}

int lobpcg_set_options(lobpcg_t* h, int tol_mode, int gram_mode, int phase_timing) {
    return guarded(h, [&] {
        LG_REQUIRE(tol_mode == LOBPCG_TOL_RELATIVE || tol_mode == LOBPCG_TOL_ABSOLUTE,
                   LOBPCG_ERR_ARG, "unknown tolerance mode");
        LG_REQUIRE(gram_mode == LOBPCG_GRAM_EXPLICIT || gram_mode == LOBPCG_GRAM_PAPER,
                   LOBPCG_ERR_ARG, "unknown Gram mode");
        h->tol_mode = tol_mode;
        h->gram_mode = gram_mode;
        h->phase_timing = phase_timing ? 1 : 0;
        return LOBPCG_OK;
    });
}

int lobpcg_set_inner_pcg(lobpcg_t* h, int iters) {
    return guarded(h, [&] {
        LG_REQUIRE(iters >= 0 && iters <= 10000, LOBPCG_ERR_ARG, "inner PCG iterations out of range [0, 10000]");
        LG_REQUIRE(iters == 0 || h->precision == LOBPCG_FP64, LOBPCG_ERR_ARG,
                   "inner PCG needs a LOBPCG_FP64 handle");
        h->inner_pcg = iters;
        return LOBPCG_OK;
    });
}

int lobpcg_set_wait_limit(lobpcg_t* h, int polls) {
    return guarded(h, [&] {
        h->wait_limit = polls < 0 ? -1 : polls;
        return LOBPCG_OK;
    });
}

int lobpcg_set_gram_engine(lobpcg_t* h, int engine) {
    return guarded(h, [&] {
        LG_REQUIRE(engine == LOBPCG_ENGINE_AUTO || engine == LOBPCG_ENGINE_TENSOR || engine == LOBPCG_ENGINE_SIMT,
                   LOBPCG_ERR_ARG,
                   "unknown Gram engine");
        h->gram_engine = engine;
        return LOBPCG_OK;
    });
}

int lobpcg_set_initial(lobpcg_t* h, const double* X0, int m, int64_t ldx, int on_host) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(X0 && m >= 1 && m <= LOBPCG_MAX_M && valid_ld(ldx, n), LOBPCG_ERR_ARG,
                   "invalid initial block");
        ensure(h, h->X0, (size_t)n * m * sizeof(double));
        LG_CUDA(cudaMemcpy2DAsync(h->X0.p, n * sizeof(double), X0, ldx * sizeof(double),
                                  n * sizeof(double), m,
                                  on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  h->stream));
        LG_CUDA(cudaStreamSynchronize(h->stream));
        h->X0_m = m;
        return LOBPCG_OK;
    });
}

int lobpcg_set_constraints(lobpcg_t* h, const double* Y, int l, int64_t ldy, int on_host) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(l >= 0 && 2 * (int64_t)l < n && (l == 0 || (Y && valid_ld(ldy, n))), LOBPCG_ERR_ARG,
                   "invalid constraint block");
        h->state = 0;      // a solve in progress used the previous constraints
        free_constraints(h);
        if (l == 0) return LOBPCG_OK;
        const int64_t ld = round_up(n, 32);          // the workspace's leading dimension
        ensure(h, h->Yq, (size_t)ld * l * sizeof(double));
        LG_CUDA(cudaMemcpy2DAsync(h->Yq.p, ld * sizeof(double), Y, ldy * sizeof(double), n * sizeof(double), l,
                                  on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
        LG_CUDA(cudaStreamSynchronize(h->stream));
        h->ncon = l;
        return LOBPCG_OK;
    });
}

int lobpcg_begin(lobpcg_t* h, int m, double tol, uint64_t seed) {
    if (h) h->launches_at_start = g_kernel_launches.load();
    return guarded(h, [&] {
        h->state = 0;
        begin(h, m, tol, seed);
        return LOBPCG_OK;
    });
}

int lobpcg_iterate(lobpcg_t* h, int steps, lobpcg_info* out) {
    if (h) h->launches_at_start = g_kernel_launches.load();
    int rc = guarded(h, [&] {
        LG_REQUIRE(h->state == 1, LOBPCG_ERR_STATE, "call lobpcg_begin first");
        LG_REQUIRE(steps >= 0, LOBPCG_ERR_ARG, "steps must be >= 0");
        int r = LOBPCG_NOT_CONVERGED;
        // `steps` passes of the iteration of Section 2.2, then the check of the pass after them
        r = run_passes(h, steps);
        return r;
    });
    if (h && out) fill_info(h, out, rc);
    return rc;
}

int lobpcg_finish(lobpcg_t* h, lobpcg_info* out) {
    int rc = guarded(h, [&] {
        LG_REQUIRE(h->state >= 1, LOBPCG_ERR_STATE, "nothing to finish");
        finish(h);
        return h->J.empty() ? LOBPCG_OK : LOBPCG_NOT_CONVERGED;
    });
    if (h && out) fill_info(h, out, rc);
    return rc;
}

int lobpcg_solve(lobpcg_t* h, int m, double tol, int maxit, uint64_t seed, lobpcg_info* out) {
    if (h) h->launches_at_start = g_kernel_launches.load();
    int rc = guarded(h, [&] {
        LG_REQUIRE(maxit >= 0, LOBPCG_ERR_ARG, "maxit must be >= 0");
        h->state = 0;
        begin(h, m, tol, seed);
        int r = LOBPCG_NOT_CONVERGED;
        try {
            r = run_passes(h, maxit);
        } catch (const Error& e) {
            if (e.code == LOBPCG_ERR_CUDA) throw;
            finish(h);   // last valid iterate stays available
            throw;
        }
        finish(h);
        return r;
    });
    if (h && out) fill_info(h, out, rc);
    return rc;
}

int lobpcg_get_eigenpairs(lobpcg_t* h, double* lambda, double* X, int64_t ldx, int x_on_host,
                          double* resid) {
    return guarded(h, [&] {
        LG_REQUIRE(h->state == 2, LOBPCG_ERR_STATE, "no finished solve on this handle");
        const int m = h->m;
        const int64_t n = h->g.n();
        if (lambda) std::memcpy(lambda, h->lam_h.data(), m * sizeof(double));
        if (resid) std::memcpy(resid, h->resid_h.data(), m * sizeof(double));
        if (X) {
            LG_REQUIRE(valid_ld(ldx, n), LOBPCG_ERR_ARG, "ldx < n");
            LG_CUDA(cudaMemcpy2DAsync(X, ldx * sizeof(double), h->X.p, h->ld * sizeof(double),
                                      n * sizeof(double), m,
                                      x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                      h->stream));
            LG_CUDA(cudaStreamSynchronize(h->stream));
        }
        return LOBPCG_OK;
    });
}

int lobpcg_eig_grad_kappa(lobpcg_t* h, const double* w, double* grad_faces) {
    return guarded(h, [&] {
        LG_REQUIRE(h->state == 2, LOBPCG_ERR_STATE, "no finished solve on this handle");
        LG_REQUIRE(h->varcoef, LOBPCG_ERR_STATE, "the operator is not LOBPCG_VARCOEF7");
        LG_REQUIRE(w && grad_faces, LOBPCG_ERR_ARG, "w and grad_faces must not be NULL");
        for (int j = 0; j < h->m; ++j) LG_REQUIRE(std::isfinite(w[j]), LOBPCG_ERR_ARG, "non-finite weight");
        launch_vc_grad(h->g, h->m, w, h->scale, f64(h->X), h->ld, grad_faces, h->stream);
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

const char* lobpcg_last_error(const lobpcg_t* h) {
    if (!h) return g_handle_free_error.c_str();
    return h->err.c_str();
}

int lobpcg_destroy(lobpcg_t* h) {
    if (!h) return LOBPCG_OK;
    cudaSetDevice(h->device);
    if (!h->poisoned) {
        free_workspace(h);
        dfree(h, h->coarse_tab);
        dfree(h, h->X0);
        dfree(h, h->pcg_small);
        free_varcoef(h);
        free_constraints(h);
        cudaStreamSynchronize(h->stream);
        for (auto& e : h->ev)
            if (e) cudaEventDestroy(e);
    }
    cudaGetLastError();
    delete h;
    return LOBPCG_OK;
}

// ---------------------------------------------------------------------- kernel-level ops
int lobpcg_op_random_block(lobpcg_t* h, uint64_t seed, int m, double* X, int64_t ldx) {
    return guarded(h, [&] {
        require_op(h);
        LG_REQUIRE(X && m >= 1 && valid_ld(ldx, h->g.n()), LOBPCG_ERR_ARG, "invalid block");
        launch_random_block(seed, h->g.n(), m, X, ldx, h->stream);
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_stencil(lobpcg_t* h, int ncols, const double* X, int64_t ldx, double* Y, int64_t ldy) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(X && Y && ncols >= 0 && valid_ld(ldx, n) && valid_ld(ldy, n), LOBPCG_ERR_ARG,
                   "invalid stencil arguments");
        spmv(h, ncols, DT_F64, X, ldx, Y, ldy);
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_stencil_f32(lobpcg_t* h, int ncols, const float* X, int64_t ldx, float* Y, int64_t ldy) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(X && Y && ncols >= 0 && valid_ld(ldx, n) && valid_ld(ldy, n), LOBPCG_ERR_ARG,
                   "invalid stencil arguments");
        LG_REQUIRE(h->precision == LOBPCG_MIXED && !h->varcoef, LOBPCG_ERR_ARG,
                   "lobpcg_op_stencil_f32 needs a LOBPCG_MIXED handle");
        spmv(h, ncols, DT_F32, X, ldx, Y, ldy);
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_precond(lobpcg_t* h, int ncols, const double* R, int64_t ldr, double* E, int64_t lde) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(R && E && ncols >= 1 && ncols <= LOBPCG_MAX_M && valid_ld(ldr, n) &&
                       valid_ld(lde, n),
                   LOBPCG_ERR_ARG, "invalid preconditioner arguments");
        LG_REQUIRE(h->precision == LOBPCG_FP64, LOBPCG_ERR_ARG,
                   "lobpcg_op_precond needs a LOBPCG_FP64 handle");
        ensure_workspace(h, std::max(h->wm, ncols));
        if (h->inner_pcg > 0) {
            copy_cols(h, ncols, n, DT_F64, R, ldr, h->W.p, h->ld);
            inner_pcg(h, ncols, f64(h->W), f64(h->E0), f64(h->Pc), f64(h->APc), f64(h->AW), f64(h->T0));
            copy_cols(h, ncols, n, DT_F64, h->E0.p, h->ld, E, lde);
        } else {
            precond(h, ncols, DT_F64, R, ldr, E, lde, h->T0.p, h->ld);
        }
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_precond_f32(lobpcg_t* h, int ncols, const float* R, int64_t ldr, float* E, int64_t lde) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(R && E && ncols >= 1 && ncols <= LOBPCG_MAX_M && valid_ld(ldr, n) && valid_ld(lde, n),
                   LOBPCG_ERR_ARG, "invalid preconditioner arguments");
        LG_REQUIRE(h->precision == LOBPCG_MIXED, LOBPCG_ERR_ARG, "lobpcg_op_precond_f32 needs a LOBPCG_MIXED handle");
        ensure_workspace(h, std::max(h->wm, ncols));
        precond(h, ncols, DT_F32, R, ldr, E, lde, h->T0.p, h->ld);
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_residual(lobpcg_t* h, int ncols, const int* cols, const double* X, const double* AX,
                       int64_t ld, const double* lambda, double* W, int64_t ldw, double* norms) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(ncols >= 1 && ncols <= LOBPCG_MAX_M && cols && X && AX && lambda && norms &&
                       valid_ld(ld, n) && (!W || valid_ld(ldw, n)),
                   LOBPCG_ERR_ARG, "invalid residual arguments");
        ensure_workspace(h, std::max(h->wm, ncols));
        ColList cl{};
        cl.n = ncols;
        for (int t = 0; t < ncols; ++t) cl.idx[t] = cols[t];
        launch_residual(n, cl, X, AX, ld, lambda, DT_F64, W, ldw, f64(h->part), h->stream);
        launch_norms_finalize(ncols, residual_chunks(n), f64(h->part), h->norms, h->stream);
        LG_CUDA(cudaMemcpyAsync(norms, h->norms, ncols * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
        LG_CUDA(cudaStreamSynchronize(h->stream));
        return LOBPCG_OK;
    });
}

int lobpcg_op_gram(lobpcg_t* h, const double* S0, const double* S1, const double* S2,
                   const double* AS0, const double* AS1, const double* AS2, int64_t ld, int w0,
                   int w1, int w2, double* gramA, double* gramB) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        const int q = w0 + w1 + w2;
        LG_REQUIRE(S0 && gramB && w0 >= 1 && w1 >= 0 && w2 >= 0 && q <= 3 * LOBPCG_MAX_M &&
                       (w1 == 0 || S1) && (w2 == 0 || S2) && valid_ld(ld, n),
                   LOBPCG_ERR_ARG, "invalid Gram arguments");
        LG_REQUIRE(!AS0 || (gramA && (w1 == 0 || AS1) && (w2 == 0 || AS2)), LOBPCG_ERR_ARG,
                   "invalid Gram arguments (A side)");
        ensure_workspace(h, std::max(h->wm, (q + 2) / 3));
        const Blocks3 S = blocks(S0, w0, DT_F64, S1, w1, S2, w2, DT_F64, ld);
        const Blocks3 AS = blocks(AS0, w0, DT_F64, AS1, w1, AS2, w2, DT_F64, ld);
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
        gram(h, S, AS0 ? &AS : nullptr, gramA, gramB, nullptr, true);
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        LG_CUDA(cudaStreamSynchronize(h->stream));
        if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
        return LOBPCG_OK;
    });
}

int lobpcg_op_gram_f32(lobpcg_t* h, const float* S0, int w0, const float* S1, int w1, const float* V, int b,
                       int64_t ld, double* C, double* G) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(V && b >= 1 && b <= LOBPCG_MAX_M_MIXED && w0 >= 0 && w1 >= 0 && w0 + w1 <= 2 * LOBPCG_MAX_M_MIXED &&
                       (w0 == 0 || S0) && (w1 == 0 || S1) && valid_ld(ld, n),
                   LOBPCG_ERR_ARG, "invalid float32 Gram arguments");
        ensure_workspace(h, std::max(h->wm, (w0 + w1 + b + 2) / 3));
        cudaStream_t st = h->stream;
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        launch_gram32_cross(n, ld, S0, w0, S1, w1, V, b, (w0 + w1) ? C : nullptr, G, f64(h->part),
                            (int64_t)h->part_doubles, h->status, use_tc(h), st);
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        LG_CUDA(cudaStreamSynchronize(st));
        if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
        return LOBPCG_OK;
    });
}

int lobpcg_op_gram_residual(lobpcg_t* h, const float* Xh, const float* Xl, const float* W, const float* P,
                            const float* R, const float* AW, const float* AP, int64_t ld, int m, int b, int bp,
                            const double* lambda, double* gramA, double* gramB) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(Xh && Xl && R && lambda && gramA && gramB && m >= 1 && m <= LOBPCG_MAX_M_MIXED && b >= 1 &&
                       b <= LOBPCG_MAX_M_MIXED && bp >= 0 && bp <= LOBPCG_MAX_M_MIXED && W && AW &&
                       (bp == 0 || (P && AP)) &&
                       valid_ld(ld, n),
                   LOBPCG_ERR_ARG, "invalid residual-form Gram arguments");
        ensure_workspace(h, std::max(h->wm, (m + b + bp + 2) / 3));
        cudaStream_t st = h->stream;
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        launch_gram_mx2(n, ld, Xh, Xl, W, bp ? P : W, R, AW, bp ? AP : AW, m, b, bp, f64(h->part),
                        (int64_t)h->part_doubles, lambda, gramA, gramB, h->status, use_tc(h), st);
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        LG_CUDA(cudaStreamSynchronize(st));
        if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
        return LOBPCG_OK;
    });
}

int lobpcg_op_cholqr(lobpcg_t* h, int b, double* V, double* AV, int64_t ld) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        LG_REQUIRE(V && b >= 1 && b <= LOBPCG_MAX_M && valid_ld(ld, n), LOBPCG_ERR_ARG,
                   "invalid CholQR arguments");
        ensure_workspace(h, std::max(h->wm, b));
        cudaStream_t st = h->stream;
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        const Blocks3 SV = blocks(V, b, DT_F64, nullptr, 0, nullptr, 0, DT_F64, ld);
        gram(h, SV, nullptr, h->gramA, h->Gsmall, nullptr, false);
        launch_chol_rinv(b, h->Gsmall, h->Rinv, h->status, ST_W_BREAKDOWN, 0u, st);
        if (ld == h->ld) {
            apply_rinv_f64(h, b, V, h->Rinv, ST_W_BREAKDOWN);
            if (AV) apply_rinv_f64(h, b, AV, h->Rinv, ST_W_BREAKDOWN);
        } else {
            launch_apply_rinv(n, b, DT_F64, V, ld, V, ld, h->Rinv, h->status, ST_W_BREAKDOWN, st);
            if (AV) launch_apply_rinv(n, b, DT_F64, AV, ld, AV, ld, h->Rinv, h->status, ST_W_BREAKDOWN, st);
        }
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        LG_CUDA(cudaStreamSynchronize(st));
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        if (stw & ST_W_BREAKDOWN) throw Error(LOBPCG_ERR_BREAKDOWN, "Gram matrix not positive definite");
        return LOBPCG_OK;
    });
}

int lobpcg_op_update(lobpcg_t* h, const double* S0, const double* S1, const double* S2, int64_t ld, int w0,
                     int w1, int w2, int m, const double* C, double* Xout, double* Pout) {
    return guarded(h, [&] {
        require_op(h);
        const int64_t n = h->g.n();
        const int q = w0 + w1 + w2;
        LG_REQUIRE(S0 && C && Xout && w0 >= 1 && w1 >= 0 && w2 >= 0 && q <= 3 * LOBPCG_MAX_M && m >= 1 &&
                       m <= LOBPCG_MAX_M && (w1 == 0 || S1) && (w2 == 0 || S2) && valid_ld(ld, n),
                   LOBPCG_ERR_ARG, "invalid update arguments");
        ensure_workspace(h, std::max(h->wm, std::max(m, (q + 2) / 3)));
        const Blocks3 S = blocks(S0, w0, DT_F64, S1, w1, S2, w2, DT_F64, ld);
        LG_CUDA(cudaMemcpyAsync(h->Cm, C, sizeof(double) * (size_t)q * m, cudaMemcpyDeviceToDevice, h->stream));
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
        h->colexp_q = 0;                 // no Gram of this basis: the plain frame per grid point
        update_f64(h, m, S, Xout, Pout, 0u, 0);
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        LG_CUDA(cudaStreamSynchronize(h->stream));
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
        if (stw & ST_TIMEOUT) throw Error(LOBPCG_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
        return LOBPCG_OK;
    });
}

int lobpcg_op_rayleigh_ritz(lobpcg_t* h, int q, int m, const double* gramA, const double* gramB,
                            double* lambda, double* C) {
    return guarded(h, [&] {
        require_op(h);
        LG_REQUIRE(gramA && gramB && lambda && C && q >= 1 && q <= 3 * LOBPCG_MAX_M && m >= 1 &&
                       m <= q,
                   LOBPCG_ERR_ARG, "invalid Rayleigh-Ritz arguments");
        ensure_workspace(h, std::max(h->wm, (q + 2) / 3));
        cudaStream_t st = h->stream;
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        launch_rayleigh_ritz(q, q, m, gramA, gramB, lambda, C, h->rrwork, h->status, 0u, st);
        unsigned stw = 0;
        LG_CUDA(cudaMemcpyAsync(&stw, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        LG_CUDA(cudaStreamSynchronize(st));
        LG_CUDA(cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
        if (stw & ST_RR_BREAKDOWN) throw Error(LOBPCG_ERR_BREAKDOWN, "gramB not positive definite");
        if (stw & ST_NONFINITE) throw Error(LOBPCG_ERR_NONFINITE, "non-finite eigenvalue");
        return LOBPCG_OK;
    });
}

}  // extern "C"
