// Double-word (FP64-class) arithmetic on the FP32 pipes for the Lanczos
// products: a value is the unevaluated sum hi + lo of two floats (about 47
// significant bits here), products are exact by FMA (p + e = a*b), sums use
// the two-sum of Knuth (the double-word algorithms of Dekker 1971 and of
// Joldes, Muller and Popescu 2017; accumulation as in Dot2 of Ogita, Rump and
// Oishi 2005).  GB300 runs FP64 at 1/64 of the FP32 rate, so products with
// several multiply-adds per element of the basis run faster this way.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ml {
namespace dword {

// FP64 -> (hi, lo) from the bits of v with integer operations only: hi keeps
// the leading 24 significant bits, lo the next 23 (relative error <= 2^-47);
// values below 2^-103 keep hi only, below 2^-126 become zero
__device__ __forceinline__ float2 from_double(double v)
{
    const uint32_t whi = (uint32_t)__double2hiint(v), wlo = (uint32_t)__double2loint(v);
    const uint32_t sgn = whi & 0x80000000u;
    const int ef = (int)((whi >> 20) & 0x7FF) - 1023 + 127;       // float exponent of hi
    if (ef <= 0) return make_float2(0.0f, 0.0f);
    const uint32_t mant = ((whi & 0xFFFFFu) << 3) | (wlo >> 29);   // top 23 mantissa bits
    const float hi = __uint_as_float(sgn | ((uint32_t)ef << 23) | mant);
    float lo = 0.0f;
    if (ef > 23) {
        // the next 23 bits under the exponent of hi minus 23, minus the implicit one
        const uint32_t base = sgn | ((uint32_t)(ef - 23) << 23);
        lo = __fsub_rn(__uint_as_float(base | ((wlo & 0x1FFFFFFFu) >> 6)), __uint_as_float(base));
    }
    return make_float2(hi, lo);
}

__device__ __forceinline__ double to_double(float2 x) { return (double)x.x + (double)x.y; }

// s += a * b, s unnormalised (s.y gathers the rounding errors of the running
// sum and of the products)
__device__ __forceinline__ void fma_acc(float2 &s, float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float t = __fadd_rn(s.x, p);
    const float bb = __fsub_rn(t, s.x);
    const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s.y = __fadd_rn(s.y, __fadd_rn(err, e));
    s.x = t;
}

}  // namespace dword
}  // namespace ml
