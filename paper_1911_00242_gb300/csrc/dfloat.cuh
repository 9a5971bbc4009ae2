// Double-float arithmetic (FP32 pairs) for the Ozaki form.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace ccsdk {

// The rounded FP32 operations the error-free transformations are written with.  On
// the device they are intrinsics, which the compiler neither contracts nor
// reassociates; a host build (the CPU tests of this arithmetic) must be compiled
// with -ffp-contract=off for the same guarantee.
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float df_add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float df_sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float df_mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float df_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float df_add_rn(float a, float b) { return a + b; }
inline float df_sub_rn(float a, float b) { return a - b; }
inline float df_mul_rn(float a, float b) { return a * b; }
inline float df_fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
#endif

// Double-float ("df") numbers for the Ozaki form's FP64-class arithmetic off the
// tensor cores (its remaining GEMMs and the t1 terms of the ladder's W'): x = h + l with
// |l| <= ulp(h) / 2, about 48 significant bits, in FP32 arithmetic (GB300's FP32 pipe
// issues about 64 times as many operations per clock as its FP64 pipe).  The
// error-free transformations are TwoSum (Knuth) and the FMA product error; the
// intrinsics keep the compiler from contracting or reassociating them.
struct df {
    float h, l;
    __host__ __device__ __forceinline__ df() {}
    __host__ __device__ __forceinline__ df(float a, float b) : h(a), l(b) {}
    __host__ __device__ __forceinline__ explicit df(int x) : h((float)x), l(0.f) {}
    __host__ __device__ __forceinline__ explicit df(float x) : h(x), l(0.f) {}
    __host__ __device__ __forceinline__ explicit df(double x) : h((float)x), l((float)(x - (double)h)) {}
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
};

__host__ __device__ __forceinline__ df df_renorm(float s, float t) {      // (s, t) -> h + l, |l| <= ulp(h) / 2
    const float h = df_add_rn(s, t);
    return df(h, df_sub_rn(t, df_sub_rn(h, s)));
}

__host__ __device__ __forceinline__ df operator+(df a, df b) {
    const float s = df_add_rn(a.h, b.h);
    const float bb = df_sub_rn(s, a.h);
    float e = df_add_rn(df_sub_rn(a.h, df_sub_rn(s, bb)), df_sub_rn(b.h, bb));
    e = df_add_rn(e, df_add_rn(a.l, b.l));
    return df_renorm(s, e);
}

__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + df(-b.h, -b.l); }

__host__ __device__ __forceinline__ df operator*(df a, df b) {
    const float p = df_mul_rn(a.h, b.h);
    float e = df_fma_rn(a.h, b.h, -p);
    e = df_fma_rn(a.h, b.l, e);
    e = df_fma_rn(a.l, b.h, e);
    return df_renorm(p, e);
}

// a * b + c
__host__ __device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = df_mul_rn(a.h, b.h);
    float e = df_fma_rn(a.h, b.h, -p);
    e = df_fma_rn(a.h, b.l, e);
    e = df_fma_rn(a.l, b.h, e);
    const float s = df_add_rn(p, c.h);
    const float bb = df_sub_rn(s, p);
    float t = df_add_rn(df_sub_rn(p, df_sub_rn(s, bb)), df_sub_rn(c.h, bb));
    t = df_add_rn(t, df_add_rn(e, c.l));
    return df_renorm(s, t);
}

using ::fma;             // the float and double overloads stay visible beside the df one

struct df2 { df x, y; };

__device__ __forceinline__ df2 ld_df2(const double2* p) { const double2 z = *p; return df2{df(z.x), df(z.y)}; }
__device__ __forceinline__ df2 ld_df2(const float2* p) { const float2 z = *p; return df2{df(z.x), df(z.y)}; }
__device__ __forceinline__ df2 ld_df2(const df2* p) { return *p; }

// dst = src as double-float pairs (the split costs FP64 operations, so constant inputs
// are converted once)
__global__ void to_df2_kernel(df2* __restrict__ dst, const double2* __restrict__ src, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = ld_df2(src + e);
}

}  // namespace ccsdk
