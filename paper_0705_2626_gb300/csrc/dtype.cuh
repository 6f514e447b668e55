// Typed loads and stores of the block storage types (float64, float32, bfloat16).
#pragma once

#include <cuda_bf16.h>

namespace lg {

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

__device__ __forceinline__ double ld_as(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_as(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_as(const __nv_bfloat16* p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ void st_as(double* p, double v) { *p = v; }
__device__ __forceinline__ void st_as(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_as(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_as(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void st_as(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }
__device__ __forceinline__ void st_as(double* p, float v) { *p = (double)v; }

}  // namespace lg
