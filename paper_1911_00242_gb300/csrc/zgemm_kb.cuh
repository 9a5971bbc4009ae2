// k-blocked batched complex GEMM (SIMT, FP64 DFMA).
//
//   C_b (+)= alpha * sum_{c < nchunk} opA(A_{b,c}) opB(B_{b,c})      b < nbatch
//
// Every contraction of the periodic CCSD residual is a sum over one
// "chunk" momentum (k_e, k_n, k_m, ...) of dense orbital contractions between
// momentum blocks whose positions follow from momentum conservation (paper
// Sec. 3.2.5).  The position of block (b, c) of each operand is an element
// offset in a device table; inside a block the element (r, s) sits at
// row_off[r] + col_off[s], which expresses any index permutation of a
// row-major orbital block (all CCSD layouts are separable that way).  This
// replaces the paper's ALLTOALL "index changes" (Sec. 4.3.3): operands are
// read in place, whatever their storage order.
//
// GB300's FP64 pipe (about 1 TFLOP/s, a 75th of its FP32 rate) is the bound:
// one 64x64x8 complex tile step is ~130k DFMA, so global loads without
// staging overlap are a rounding error and tiles are chosen to waste as few
// DFMAs on padding as possible.
//
// The kernel is instantiated for two arithmetic types: double (the FP64 form)
// and float (the mixed form's CUDA-core contractions: operands are read from
// complex64 copies where the plan has them, otherwise rounded from complex128
// on load; products accumulate in FP32 and the epilogue adds alpha * acc into
// the FP64 result).  Integrals stored complex64 are read through A32/B32 by
// both; the double instance widens them exactly.  On GB300 a double->float conversion issues on the slow
// FP64 pipe, so the complex64 copies matter for throughput, not only bytes.
#pragma once
#include "dfloat.cuh"
#include "tf32_split.cuh"
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccsdk {

struct GemmArgs {
    const double2* A; const long long* offA; const int* rowA; const int* colA;
    const double2* B; const long long* offB; const int* rowB; const int* colB;
    const float2* A32; const float2* B32;   // complex64 A / B (copies, or inputs stored so), used instead when set
    double2* C;       const long long* offC; const int* rowC; const int* colC;
    double2* work;    // split partials [nsplit][nbatch][M*N] when nsplit > 1
    const int* nchunk_b;   // per-batch chunk count (<= nchunk), or null for nchunk everywhere
    // antisymmetric mirror: each result is also subtracted at offC2[b] + rowC[m] + colC2[n]
    const long long* offC2; const int* colC2;
    int M, N, K, nbatch, nchunk, nsplit, chunks_per_split;
    int conjA, conjB, accumulate;
    double alpha_re, alpha_im;
    int tiles_m, tiles_n;
    // Affine operand tables (set on the host when every entry fits): element (m, k) of A
    // at offA + a0 + m * rAs + k * cAs, element (k, n) of B at offB + b0 + k * rBs + n * cBs.
    // Gathers then skip the table loads, and an operand whose K index is contiguous is
    // staged K-fastest (consecutive threads read consecutive elements).
    int affA, affB;
    long long a0, b0;
    int rAs, cAs, rBs, cBs;
};

template <typename T> struct Cplx;
template <> struct Cplx<double> { using V = double2; };
template <> struct Cplx<float> { using V = float2; };
template <> struct Cplx<df> { using V = df2; };

// A complex128 operand element in the instance's arithmetic.  The FP32 instance rounds
// with integer operations (f32_rn; the double-float conversion does the same itself):
// on GB300 every FP64 operation, a conversion included, issues on a pipe of 2 per clock
// and SM.  The results are those of the plain conversions, bit for bit.
template <typename T> __device__ __forceinline__ T from_f64(double x) { return T(x); }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return f32_rn(x); }


// Shared-memory staging of one K step: the complex tiles, and for the FP64
// instance also Re + Im of every element (the third factor of the 3M product).
template <int BM, int BN, int BK, typename T>
struct ZgemmSmem {
    typename Cplx<T>::V A[BK][BM];
    typename Cplx<T>::V B[BK][BN];
    T As[BK][BM];
    T Bs[BK][BN];
};

// One output tile (tile, batch b, K split) of one GEMM; called by the plain
// kernel below and by the grouped persistent kernel of the batched form.
//
// FP64 instance: 3M complex products.  With a = ar + i ai, b = br + i bi,
//   t1 = sum ar br,  t2 = sum ai bi,  t3 = sum (ar + ai)(br + bi),
//   Re c = t1 - t2,  Im c = t3 - t1 - t2,
// three FP64 FMAs per complex multiply-add instead of four (the sums ar + ai
// and br + bi are formed once per element when the tile is staged).  The FP32
// instance keeps the four-product form, whose imaginary part has no
// cancellation (its operands are already rounded to FP32).
//
// KS > 1 (skinny contractions: few outputs, long K): the CTA's threads form KS groups
// of (BM / TM) (BN / TN) threads; all of them stage each K step, group q multiplies
// its BK / KS rows of it, and at the end the groups' partial sums are added in group
// order (deterministic) before the epilogue.  A tile then keeps KS times more
// independent accumulators and loads in flight per barrier.
template <int BM, int BN, int BK, int TM, int TN, typename T, int KS = 1>
__device__ __forceinline__ void zgemm_tile(const GemmArgs& g, int tile, long long b, int split,
                                           ZgemmSmem<BM, BN, BK, T>& sm)
{
    using V = typename Cplx<T>::V;
    constexpr bool k3M = sizeof(T) == 8;         // double and double-float: 3M products
    constexpr int NT1 = (BM / TM) * (BN / TN);   // threads of one K group
    constexpr int NT = NT1 * KS;
    constexpr int TX = BN / TN;
    constexpr int KG = BK / KS;                  // K rows of a stage per group
    static_assert(BK % KS == 0, "each K group takes an equal share of a stage");
    const int m0 = (tile % g.tiles_m) * BM;
    const int n0 = (tile / g.tiles_m) * BN;
    const int tid = threadIdx.x;
    const int kgrp = tid / NT1;
    const int tx = (tid % NT1) % TX, ty = (tid % NT1) / TX;
    auto& As = sm.A;
    auto& Bs = sm.B;

    // 4M: (cr, ci); 3M: (cr, ci, cs) = (t1, t2, t3)
    T cr[TM][TN], ci[TM][TN], cs[TM][k3M ? TN : 1];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            cr[i][j] = T(0); ci[i][j] = T(0);
            if (k3M) cs[i][k3M ? j : 0] = T(0);
        }

    const T sa = g.conjA ? T(-1) : T(1);
    const T sb = g.conjB ? T(-1) : T(1);
    const int c_begin = split * g.chunks_per_split;
    int c_end = c_begin + g.chunks_per_split;
    const int nch = g.nchunk_b ? g.nchunk_b[b] : g.nchunk;
    if (c_end > nch) c_end = nch;

    for (int c = c_begin; c < c_end; ++c) {
        const long long oa = g.offA[b * g.nchunk + c];
        const long long ob = g.offB[b * g.nchunk + c];
        const float2* Ab32 = g.A32 ? g.A32 + oa : nullptr;
        const float2* Bb32 = g.B32 ? g.B32 + ob : nullptr;
        const double2* Ab = Ab32 ? nullptr : g.A + oa;
        const double2* Bb = Bb32 ? nullptr : g.B + ob;
        const bool kfA = g.affA && g.cAs == 1, kfB = g.affB && g.rBs == 1;
        for (int k0 = 0; k0 < g.K; k0 += BK) {
            for (int e = tid; e < BM * BK; e += NT) {
                const int mm = kfA ? e / BK : e % BM, kk = kfA ? e % BK : e / BM;
                const int m = m0 + mm, k = k0 + kk;
                V v; v.x = T(0); v.y = T(0);
                if (m < g.M && k < g.K) {
                    const long long q = g.affA ? g.a0 + (long long)m * g.rAs + (long long)k * g.cAs
                                               : (long long)g.rowA[m] + g.colA[k];
                    if (Ab32) { const float2 w = __ldg(Ab32 + q); v.x = T(w.x); v.y = T(w.y) * sa; }
                    else { const double2 w = __ldg(Ab + q); v.x = from_f64<T>(w.x); v.y = from_f64<T>(w.y) * sa; }
                }
                As[kk][mm] = v;
                if (k3M) sm.As[kk][mm] = v.x + v.y;
            }
            for (int e = tid; e < BN * BK; e += NT) {
                const int nn = kfB ? e / BK : e % BN, kk = kfB ? e % BK : e / BN;
                const int n = n0 + nn, k = k0 + kk;
                V v; v.x = T(0); v.y = T(0);
                if (n < g.N && k < g.K) {
                    const long long q = g.affB ? g.b0 + (long long)k * g.rBs + (long long)n * g.cBs
                                               : (long long)g.rowB[k] + g.colB[n];
                    if (Bb32) { const float2 w = __ldg(Bb32 + q); v.x = T(w.x); v.y = T(w.y) * sb; }
                    else { const double2 w = __ldg(Bb + q); v.x = from_f64<T>(w.x); v.y = from_f64<T>(w.y) * sb; }
                }
                Bs[kk][nn] = v;
                if (k3M) sm.Bs[kk][nn] = v.x + v.y;
            }
            __syncthreads();
#pragma unroll
            for (int kq = 0; kq < KG; ++kq) {
                const int kk = kgrp * KG + kq;
                V a[TM], bb[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
                for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx * TN + j];
                if (k3M) {
                    T sa[TM], sb[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) sa[i] = sm.As[kk][ty * TM + i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) sb[j] = sm.Bs[kk][tx * TN + j];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) {
                            cr[i][j] = fma(a[i].x, bb[j].x, cr[i][j]);
                            ci[i][j] = fma(a[i].y, bb[j].y, ci[i][j]);
                            cs[i][k3M ? j : 0] = fma(sa[i], sb[j], cs[i][k3M ? j : 0]);
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) {
                            cr[i][j] = fma(a[i].x, bb[j].x, cr[i][j]);
                            cr[i][j] = fma(-a[i].y, bb[j].y, cr[i][j]);
                            ci[i][j] = fma(a[i].x, bb[j].y, ci[i][j]);
                            ci[i][j] = fma(a[i].y, bb[j].x, ci[i][j]);
                        }
                }
            }
            __syncthreads();
        }
    }

    if constexpr (KS > 1) {
        // the groups' partial sums, added in group order by group 0 (the stage buffers
        // are free: the last K step ended with a barrier)
        constexpr int NV = TM * TN * (k3M ? 3 : 2);
        static_assert(sizeof(ZgemmSmem<BM, BN, BK, T>) >= sizeof(T) * NV * NT1 * (KS > 1 ? KS - 1 : 1),
                      "the partial sums of the K groups fit the stage buffers");
        T* red = (T*)&sm;
        const int t1 = tid % NT1;
        if (kgrp > 0) {
            T* dst = red + ((long long)(kgrp - 1) * NT1 + t1) * NV;
            int q = 0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    dst[q++] = cr[i][j];
                    dst[q++] = ci[i][j];
                    if (k3M) dst[q++] = cs[i][k3M ? j : 0];
                }
        }
        __syncthreads();
        if (kgrp > 0) return;
        for (int gq = 1; gq < KS; ++gq) {
            const T* src = red + ((long long)(gq - 1) * NT1 + t1) * NV;
            int q = 0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    cr[i][j] = cr[i][j] + src[q++];
                    ci[i][j] = ci[i][j] + src[q++];
                    if (k3M) cs[i][k3M ? j : 0] = cs[i][k3M ? j : 0] + src[q++];
                }
        }
    }
    if (k3M) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const T t1 = cr[i][j], t2 = ci[i][j];
                cr[i][j] = t1 - t2;
                ci[i][j] = cs[i][k3M ? j : 0] - t1 - t2;
            }
    }
    if (g.nsplit > 1) {
        double2* W = g.work + ((long long)split * g.nbatch + b) * (long long)g.M * g.N;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int m = m0 + ty * TM + i, n = n0 + tx * TN + j;
                if (m < g.M && n < g.N) W[(long long)m * g.N + n] = make_double2((double)cr[i][j], (double)ci[i][j]);
            }
        return;
    }
    double2* Cb = g.C + g.offC[b];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int m = m0 + ty * TM + i, n = n0 + tx * TN + j;
            if (m < g.M && n < g.N) {
                double2* p = Cb + (long long)g.rowC[m] + g.colC[n];
                const double xr = (double)cr[i][j], xi = (double)ci[i][j];
                const double re = g.alpha_re * xr - g.alpha_im * xi;
                const double im = g.alpha_re * xi + g.alpha_im * xr;
                if (g.accumulate) { double2 o = *p; o.x += re; o.y += im; *p = o; }
                else *p = make_double2(re, im);
                if (g.offC2) {
                    double2* q = g.C + g.offC2[b] + (long long)g.rowC[m] + g.colC2[n];
                    double2 o = *q; o.x -= re; o.y -= im; *q = o;
                }
            }
        }
}

template <int BM, int BN, int BK, int TM, int TN, typename T = double, int KS = 1>
__global__ void __launch_bounds__((BM / TM) * (BN / TN) * KS)
zgemm_kb_kernel(const GemmArgs g)
{
    __shared__ ZgemmSmem<BM, BN, BK, T> sm;
    const int ntile = g.tiles_m * g.tiles_n;
    zgemm_tile<BM, BN, BK, TM, TN, T, KS>(g, blockIdx.x % ntile, blockIdx.x / ntile, blockIdx.y, sm);
}

// Grouped persistent form (batched solves): one launch covers the same plan
// step of many independent problems.  Work item w of the flattened list
// [member][split][batch][tile] maps to member i with prefix[i] <= w < prefix[i+1];
// every CTA strides through the list.  All members use this launch's tile shape.
template <int BM, int BN, int BK, int TM, int TN, typename T = double, int KS = 1>
__global__ void __launch_bounds__((BM / TM) * (BN / TN) * KS)
zgemm_grouped_kernel(const GemmArgs* __restrict__ gs, const long long* __restrict__ prefix, int nmem, long long total)
{
    __shared__ ZgemmSmem<BM, BN, BK, T> sm;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = nmem - 1;
        while (lo < hi) {                       // last member whose prefix <= w
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid; else hi = mid - 1;
        }
        const GemmArgs g = gs[lo];
        const long long local = w - prefix[lo];
        const long long ntile = (long long)g.tiles_m * g.tiles_n;
        const long long per_split = ntile * g.nbatch;
        const int split = (int)(local / per_split);
        const long long r = local % per_split;
        zgemm_tile<BM, BN, BK, TM, TN, T, KS>(g, (int)(r % ntile), r / ntile, split, sm);
        if (KS > 1) __syncthreads();        // the next item reuses the stage buffers
    }
}

// Deterministic split-K reduction: C_b (+)= alpha * sum_s work[s][b] in split order.
struct SplitReduceOp {
    GemmArgs g;
    __device__ void run(long long vb, long long nvb) const {
        const long long total = (long long)g.nbatch * g.M * g.N;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long b = e / ((long long)g.M * g.N);
            const int mn = (int)(e % ((long long)g.M * g.N));
            const int m = mn / g.N, n = mn % g.N;
            double re = 0.0, im = 0.0;
            for (int s = 0; s < g.nsplit; ++s) {
                const double2 w = g.work[((long long)s * g.nbatch + b) * (long long)g.M * g.N + mn];
                re += w.x; im += w.y;
            }
            double2* p = g.C + g.offC[b] + (long long)g.rowC[m] + g.colC[n];
            const double r2 = g.alpha_re * re - g.alpha_im * im;
            const double i2 = g.alpha_re * im + g.alpha_im * re;
            if (g.accumulate) { double2 o = *p; o.x += r2; o.y += i2; *p = o; }
            else *p = make_double2(r2, i2);
            if (g.offC2) {
                double2* q = g.C + g.offC2[b] + (long long)g.rowC[m] + g.colC2[n];
                double2 o = *q; o.x -= r2; o.y -= i2; *q = o;
            }
        }
    }
};
__global__ void zgemm_split_reduce(const GemmArgs g) { SplitReduceOp{g}.run(blockIdx.x, gridDim.x); }

}  // namespace ccsdk
