// lobpcg_gram_noalloc: the Gram-matrix computation of lobpcg_op_gram for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc (or any allocator) is off limits -- a host
// callback or signal handler, an embedding that owns every byte of device memory through its
// own pool and forbids the libraries it calls from allocating, a real-time loop where an
// allocation could block, or a caller without a handle (creating a handle allocates its
// workspace).  Those callers still pass their own inputs and outputs; the only memory this entry
// point needs beyond them is the per-block partial sums of the Gram kernel, and those live in
// the fixed array below, which every GPU that loads this library holds until the process exits.
//
// Contract:
//  * Scratch capacity: kNoAllocScratchDoubles doubles (8 MiB).  The number of partial sums is
//    chosen to fit (at least one), so every basis width q = w0 + w1 + w2 <= 96 fits; wider bases
//    are rejected with LOBPCG_ERR_ARG.
//  * No cudaMalloc, cudaFree or other allocating call is made, here or in what this calls.
//  * The first call on a device looks up the device address of the array (cudaGetSymbolAddress
//    with that device current) and caches it; make that first call before any stream capture.
//  * All calls share the one array and it keeps the previous call's contents.  Every partial sum
//    a call reads is written earlier by the same call, so nothing needs clearing; but two calls
//    whose kernels overlap on the GPU (different streams or threads without ordering) race on
//    the array and give wrong results.  Order them, e.g. on one stream.
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"

namespace lg {
// Error text of the handle-free entry points, returned by lobpcg_last_error(NULL).
extern thread_local std::string g_handle_free_error;
}

namespace {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;   // 8 MiB
constexpr int kNoAllocMaxQ = 96;                                 // widest basis q
constexpr int kMaxDevices = 64;

// The scratch array.  In host code `g_gram_scratch` is a host-side stand-in, not a device
// address: kernels get the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(double** out, std::string& err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return LOBPCG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device index out of range";
        return LOBPCG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LOBPCG_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LOBPCG_OK;
}

}  // namespace

extern "C" int lobpcg_gram_noalloc(const double* S0, const double* S1, const double* S2,
                                   const double* AS0, const double* AS1, const double* AS2,
                                   int64_t n, int64_t ld, int w0, int w1, int w2, double* gramA,
                                   double* gramB, void* stream) {
    using namespace lg;
    std::string& err = g_handle_free_error;
    err.clear();
    const int q = w0 + w1 + w2;
    if (!S0 || !gramB || n < 1 || ld < n || w0 < 1 || w1 < 0 || w2 < 0 || (w1 && !S1) ||
        (w2 && !S2) || (AS0 && (!gramA || (w1 && !AS1) || (w2 && !AS2)))) {
        err = "lobpcg_gram_noalloc: invalid arguments";
        return LOBPCG_ERR_ARG;
    }
    if (q > kNoAllocMaxQ || (size_t)2 * q * q > kNoAllocScratchDoubles) {
        err = "lobpcg_gram_noalloc: basis width q = " + std::to_string(q) +
              " exceeds the maximum of 96 columns";
        return LOBPCG_ERR_ARG;
    }
    double* scratch = nullptr;
    const int rc = scratch_address(&scratch, err);
    if (rc != LOBPCG_OK) return rc;
    const int nparts = (int)std::max<int64_t>(
        1, std::min<int64_t>(gram_parts(n, q), (int64_t)(kNoAllocScratchDoubles / (2 * (size_t)q * q))));
    try {
        Blocks3 S{};
        S.p[0] = S0; S.w[0] = w0;
        S.p[1] = w1 ? S1 : S0; S.w[1] = w1;
        S.p[2] = w2 ? S2 : S0; S.w[2] = w2;
        S.ld = ld;
        Blocks3 AS = S;
        if (AS0) {
            AS.p[0] = AS0;
            AS.p[1] = w1 ? AS1 : AS0;
            AS.p[2] = w2 ? AS2 : AS0;
        }
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        launch_gram(n, S, AS0 ? &AS : nullptr, scratch, nparts, st);
        launch_gram_finalize(q, nparts, scratch, AS0 != nullptr, gramA, gramB, nullptr, &S, st);
    } catch (const Error& e) {
        err = e.what();
        return e.code;
    }
    return LOBPCG_OK;
}
