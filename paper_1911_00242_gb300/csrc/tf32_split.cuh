// Split of the mixed form's operands into TF32-exact big + small parts.  Bit
// operations and FP32/FP64 arithmetic only, host-callable as well, so that the CPU
// tests check this code itself (a host build must use -ffp-contract=off).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace ccsdk {

#ifdef __CUDA_ARCH__
__device__ __forceinline__ uint32_t tf32_bits_of(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float tf32_float_of(uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ uint64_t tf32_bits64_of(double x) { return (uint64_t)__double_as_longlong(x); }
#else
inline uint32_t tf32_bits_of(float x) { uint32_t u; memcpy(&u, &x, sizeof u); return u; }
inline float tf32_float_of(uint32_t u) { float x; memcpy(&x, &u, sizeof x); return x; }
inline uint64_t tf32_bits64_of(double x) { uint64_t u; memcpy(&u, &x, sizeof u); return u; }
#endif

// A double rounded to float (round to nearest, ties to even; IEEE 754) from its bit
// pattern with integer operations, and the rounding residual x - f as a float.  On
// GB300 every FP64 operation, a conversion included, issues on a pipe of 2 per clock
// and SM, so the operand preparation avoids them.  Covers 2^-74 <= |x| < 2^127, where
// f is a normal float and the residual's scale 2^(E - 52) a normal power of two;
// returns false for every other x (zero included), which then takes the FP64 path.
__host__ __device__ __forceinline__ bool f32_round_with_residual(double x, float& f, float& r) {
    const uint64_t u = tf32_bits64_of(x);
    const int e = (int)((u >> 52) & 0x7ff);                 // biased exponent of x
    if (e < 949 || e > 1149) return false;
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const uint64_t m = u & 0xFFFFFFFFFFFFFull;                // 52 stored mantissa bits
    const uint32_t keep = (uint32_t)(m >> 29);                // the float's 23 stored bits
    const int32_t rem = (int32_t)(m & 0x1FFFFFFFull);         // the 29 dropped bits
    const bool up = rem > 0x10000000 || (rem == 0x10000000 && (keep & 1u));
    // biased float exponent e - 1023 + 127; a carry out of the mantissa bumps it (exact)
    f = tf32_float_of(sign | ((((uint32_t)(e - 896)) << 23) + keep + (up ? 1u : 0u)));
    // x - f = +-(rem - up 2^29) 2^(e - 1075): a 30-bit integer (one FP32 rounding) times a
    // power of two, with the sign of x
    const float scale = tf32_float_of(((uint32_t)(e - 948)) << 23);   // 2^(e - 1075)
    const int32_t d = up ? rem - 0x20000000 : rem;
    const float units = (float)(sign ? -d : d);                // +0 when x = f, as x - f
    r = units * scale;
    return true;
}

__host__ __device__ __forceinline__ float tf32_round(float x) {
    // round to nearest (ties away) at the 10-bit TF32 mantissa; TF32 MMAs then
    // use these values exactly
    uint32_t u = tf32_bits_of(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    return tf32_float_of(u);
}

// Split of a float into TF32-exact big + small parts (FP32 arithmetic only).
__host__ __device__ __forceinline__ void split_tf32f(float x, float& big, float& small) {
    big = tf32_round(x);
    small = tf32_round(x - big);
}

// Split of a double into TF32-exact big + small parts: big from the float rounding f
// of x, small from the remainder x - big = (f - big) + (x - f), whose first term is
// exact in FP32 and whose second is the float residual (FP32 operations only; outside
// the range of f32_round_with_residual, FP64 arithmetic).
__host__ __device__ __forceinline__ void split_tf32(double x, float& big, float& small) {
    float f, r;
    if (f32_round_with_residual(x, f, r)) {
        big = tf32_round(f);
        small = tf32_round((f - big) + r);
        return;
    }
    const float f64 = (float)x;
    big = tf32_round(f64);
    small = tf32_round((float)(x - (double)big));
}

// A double rounded to float, by integer operations where f32_round_with_residual covers x.
__host__ __device__ __forceinline__ float f32_rn(double x) {
    float f, r;
    return f32_round_with_residual(x, f, r) ? f : (float)x;
}

}  // namespace ccsdk
