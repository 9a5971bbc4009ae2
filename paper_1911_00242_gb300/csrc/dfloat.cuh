// Double-float arithmetic (FP32 pairs) for the Ozaki form.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace ccsdk {

// Double-float ("df") numbers for the Ozaki form's FP64-class arithmetic off the
// tensor cores (its remaining GEMMs and the t1 terms of the ladder's W'): x = h + l with
// |l| <= ulp(h) / 2, about 48 significant bits, in FP32 arithmetic (GB300's FP32 pipe
// issues about 64 times as many operations per clock as its FP64 pipe).  The
// error-free transformations are TwoSum (Knuth) and the FMA product error; the
// intrinsics keep the compiler from contracting or reassociating them.
struct df {
    float h, l;
    __device__ __forceinline__ df() {}
    __device__ __forceinline__ df(float a, float b) : h(a), l(b) {}
    __device__ __forceinline__ explicit df(int x) : h((float)x), l(0.f) {}
    __device__ __forceinline__ explicit df(float x) : h(x), l(0.f) {}
    __device__ __forceinline__ explicit df(double x) : h((float)x), l((float)(x - (double)h)) {}
    __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df df_renorm(float s, float t) {      // (s, t) -> h + l, |l| <= ulp(h) / 2
    const float h = __fadd_rn(s, t);
    return df(h, __fsub_rn(t, __fsub_rn(h, s)));
}

__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df_renorm(s, e);
}

__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }
__device__ __forceinline__ df operator-(df a, df b) { return a + df(-b.h, -b.l); }

__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_renorm(p, e);
}

// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float s = __fadd_rn(p, c.h);
    const float bb = __fsub_rn(s, p);
    float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.h, bb));
    t = __fadd_rn(t, __fadd_rn(e, c.l));
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
