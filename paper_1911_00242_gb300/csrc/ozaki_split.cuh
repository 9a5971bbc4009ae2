// Error-free splitting of the Ozaki form's operands into BF16 integer slices
// (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59 (2012) 95-118): the row scale,
// the fixed-point conversion and the balanced base-128 digits.  Host-callable as
// well, so that the CPU tests check this code itself; the device build uses the
// CUDA bit-cast and conversion intrinsics, the host build their exact equivalents.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <math.h>

namespace ccsdk {

constexpr int OZ_SLICE_BITS = 7;
constexpr int OZ_MAX_SLICES = 8;
constexpr int OZ_EXP_MIN = -120;                           // row-scale exponent clamp (see oz_row_exponent)
constexpr int OZ_EXP_MAX = 120;

#ifdef __CUDA_ARCH__
__device__ __forceinline__ long long oz_bits_of(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double oz_double_of(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ uint32_t oz_bits_of(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float oz_float_of(int b) { return __int_as_float(b); }
__device__ __forceinline__ long long oz_rint_ll(double x) { return __double2ll_rn(x); }
#else
inline long long oz_bits_of(double x) { long long b; memcpy(&b, &x, sizeof b); return b; }
inline double oz_double_of(long long b) { double x; memcpy(&x, &b, sizeof x); return x; }
inline uint32_t oz_bits_of(float x) { uint32_t b; memcpy(&b, &x, sizeof b); return b; }
inline float oz_float_of(int b) { float x; memcpy(&x, &b, sizeof x); return x; }
inline long long oz_rint_ll(double x) { return llrint(x); }     // the default mode: to nearest, ties to even
#endif

// Row maxima are taken on the bit patterns: for non-negative doubles the unsigned
// order of the patterns is the numeric order, and the integer pipes are far faster
// than GB300's FP64 pipe.
__host__ __device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)oz_bits_of(x) & 0x7fffffffffffffffULL;
}

// Power-of-two scale exponent E with 2^E > amax (the frexp exponent of amax, from
// its bit pattern), clamped to [OZ_EXP_MIN, OZ_EXP_MAX] so that 2^E and 1 / 2^E are
// FP32 values: rows whose largest element lies outside about 1e-36 .. 1e36 lose
// relative precision.  0 for an all-zero row.
__host__ __device__ __forceinline__ int oz_row_exponent(unsigned long long amax_bits) {
    if (amax_bits == 0) return 0;
    const int e = (int)(amax_bits >> 52) - 1022;        // biased exponent (0: subnormal) - 1022
    return e < OZ_EXP_MIN ? OZ_EXP_MIN : (e > OZ_EXP_MAX ? OZ_EXP_MAX : e);
}

// The s slices of x 2^-E, from the 7s-bit fixed point Y = rint(x 2^{7s-E}) (|Y| <= 2^{7s};
// `scale` = 2^{7s-E}, so x * scale is exact): balanced base-128 digits from the least
// significant (in [-64, 63]), the remaining top digit (|v_0| <= 128) last.  Then
// x = 2^E sum_p v_p 2^{-7(p+1)} up to 2^{E-7s-1}.  Integer arithmetic only after the
// one conversion.  Output: BF16 bit patterns (the values are integers of at most 8
// bits, so the upper half of their FP32 pattern is exact).
__host__ __device__ __forceinline__ void oz_split(double x, double scale, int s, uint16_t* out) {
    long long Y = oz_rint_ll(x * scale);
    for (int p = s - 1; p > 0; --p) {
        const int dg = (int)((Y + 64) & 127) - 64;
        Y = (Y - dg) >> 7;
        out[p] = (uint16_t)(oz_bits_of((float)dg) >> 16);
    }
    out[0] = (uint16_t)(oz_bits_of((float)(int)Y) >> 16);
}

// 2^{7s-E} as a double and 2^E as a float.
__host__ __device__ __forceinline__ double oz_fixed_scale(int s, int E) {
    return oz_double_of((long long)(1023 + OZ_SLICE_BITS * s - E) << 52);
}
__host__ __device__ __forceinline__ float oz_row_scale(int E) {
    return oz_float_of((127 + E) << 23);
}

}  // namespace ccsdk
