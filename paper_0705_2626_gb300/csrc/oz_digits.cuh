// Signed 7-bit digits of a float64 value in a given exponent frame, for the error-free digit
// products on the tensor cores (k_gram_oz.cu, k_tsmm_oz.cu).
//
// In the frame of the exponent field emax (emax >= the exponent field of x, E = emax - 1022,
// so |x| < 2^E), F = round(|x| 2^(56 - E)) is a 56-bit integer and
//     x = sign(x) 2^(E - 56) sum_{s=0..7} u_s 2^(7 (7 - s)) + err,   |err| <= 2^(E - 57),
// with u_s = bits 49 - 7 s .. 55 - 7 s of F.  The digits d_s = sign(x) u_s are exact in
// float32 and in bfloat16 (|d_s| <= 127).
//
// F is cut into four 14-bit quarters; each quarter Q goes into the low mantissa bits of the
// float32 2^23 + Q, and its two digits come out of the FMA pipe: floor(Q / 128) from one fused
// multiply-add rounded toward zero (2^23 + Q / 128 lies in [2^23, 2^24), where float32 steps
// by 1), Q mod 128 = Q - 128 floor(Q / 128) exactly; the sign enters as a factor of +-1 in the
// same fused multiply-adds.  This keeps the integer pipe to the exponent, the rounding shift and
// the quarter extraction.
#pragma once
#include <cstdint>

namespace lg {

__device__ __forceinline__ void oz_digits(double x, int emax, float (&d)[8]) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7FFu);
    const int sh = emax - e;
    // |x| 2^(56 - E) = M3 2^-sh, rounded to nearest (no branch: sh is clamped, the zero and
    // far-below-frame cases are selected away)
    const uint64_t M3 = ((((uint64_t)((hi & 0xFFFFFu) | 0x100000u)) << 32) | lo) << 3;
    const int s = min(max(sh, 0), 63);
    uint64_t F = (M3 + ((1ull << s) >> 1)) >> s;
    F = (e == 0 || sh >= 60) ? 0ull : F;
    const uint32_t fh = (uint32_t)(F >> 32), fl = (uint32_t)F;
    const float sg = __uint_as_float((hi & 0x80000000u) | 0x3F800000u);   // sign(x) as +-1
    const float nb = -8388608.0f * sg;                                    // -2^23 sign(x)
    const uint32_t magic = 0x4B000000u;                                   // 2^23
    const uint32_t q[4] = {(fh >> 10) | magic, (__funnelshift_r(fl, fh, 28) & 0x3FFFu) | magic,
                           ((fl >> 14) & 0x3FFFu) | magic, (fl & 0x3FFFu) | magic};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float X = __uint_as_float(q[k]);                       // 2^23 + Q
        const float t = __fmaf_rz(X, 0.0078125f, 8323072.0f);        // 2^23 + floor(Q / 128)
        const float h = fmaf(t, sg, nb);                             // sign * floor(Q / 128)
        const float v = fmaf(X, sg, nb);                             // sign * Q
        d[2 * k] = h;
        d[2 * k + 1] = fmaf(h, -128.0f, v);                          // sign * (Q mod 128)
    }
}

// Two float32 values with at most 8 significant bits each (exact in bfloat16) as a bfloat16
// pair: a in the low half, b in the high half.
__device__ __forceinline__ uint32_t oz_pack2(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

}  // namespace lg
