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
#else
inline uint32_t tf32_bits_of(float x) { uint32_t u; memcpy(&u, &x, sizeof u); return u; }
inline float tf32_float_of(uint32_t u) { float x; memcpy(&x, &u, sizeof x); return x; }
#endif

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

// Split of a double into TF32-exact big + small parts.
__host__ __device__ __forceinline__ void split_tf32(double x, float& big, float& small) {
    const float f = (float)x;
    big = tf32_round(f);
    small = tf32_round((float)(x - (double)big));
}

}  // namespace ccsdk
