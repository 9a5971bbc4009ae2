// Elementwise and reduction kernels of the CCSD iteration (FP64).
//
// Layout conventions (row-major, complex interleaved):
//   t1/R1  [k][i][a]               t2/R2/tau  [ki][kj][ka][i][j][a][b], kb implied
// `kb_of[(ki*N + kj)*N + ka]` is the fourth momentum of a doubles block,
// `neg` tables are not needed: every map below is precomputed on the host.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"
#include "diis.h"

namespace ccsdk {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Loads of an input element stored complex128 or complex64 (widened exactly).
__device__ __forceinline__ double2 ldz(const double2* p) { return *p; }
__device__ __forceinline__ double2 ldz(const float2* p) { const float2 f = *p; return make_double2(f.x, f.y); }

// tau~ = t2 + 1/2 x and tau = t2 + x with
// x = delta(ki,ka) t_i^a t_j^b - delta(ki,kb) t_i^b t_j^a
// (paper Sec. 2: 1/4 and 1/2 of P(ab)P(ij) t1 t1, whose four terms pair up).
// Mixed form: t2_32 / taut_32 (when set) receive complex64 copies of t2 and tau~
// for the FP32 contractions (a double->float conversion issues on GB300's FP64
// pipe, so each element is converted once here instead of in every GEMM).
struct TauOp {
    const double2* t1; const double2* t2;
    double2* tau; double2* taut;
    const int* kb_of; int N, o, v;
    float2* t2_32; float2* taut_32;
    // vb, nvb: this block's index and the block count of its (virtual) grid
    __device__ void run(long long vb, long long nvb) const {
        const long long blk = (long long)o * o * v * v;
        const long long total = (long long)N * N * N * blk;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long kk = e / blk;
            int r = (int)(e % blk);
            const int b = r % v; r /= v;
            const int a = r % v; r /= v;
            const int j = r % o; const int i = r / o;
            const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
            const int kb = kb_of[kk];
            double2 x = make_double2(0.0, 0.0);
            if (ki == ka) {
                const double2 p = cmul(t1[((long long)ki * o + i) * v + a], t1[((long long)kj * o + j) * v + b]);
                x.x += p.x; x.y += p.y;
            }
            if (ki == kb) {
                const double2 p = cmul(t1[((long long)ki * o + i) * v + b], t1[((long long)kj * o + j) * v + a]);
                x.x -= p.x; x.y -= p.y;
            }
            const double2 t = t2[e];
            tau[e] = make_double2(t.x + x.x, t.y + x.y);
            const double2 tt = make_double2(t.x + 0.5 * x.x, t.y + 0.5 * x.y);
            taut[e] = tt;
            if (t2_32) {
                t2_32[e] = make_float2((float)t.x, (float)t.y);
                taut_32[e] = make_float2((float)tt.x, (float)tt.y);
            }
        }
    }
};
__global__ void tau_kernel(const TauOp op) { op.run(blockIdx.x, gridDim.x); }

// dst = conj(src) or dst = src, n elements; src is complex128, or complex64 (src32 set)
struct CopyOp {
    double2* dst; const double2* src; const float2* src32; long long n; int conj;
    __device__ void run(long long vb, long long nvb) const {
        for (long long e = vb * blockDim.x + threadIdx.x; e < n; e += nvb * blockDim.x) {
            double2 s = src32 ? ldz(src32 + e) : ldz(src + e);
            if (conj) s.y = -s.y;
            dst[e] = s;
        }
    }
};
__global__ void copy_kernel(const CopyOp op) { op.run(blockIdx.x, gridDim.x); }

// Batched 4-index permuted copy:
//   dst[offD[b] + i0*d0 + i1*d1 + i2*d2 + i3*d3] = src[offS[b] + i0*s0 + i1*s1 + i2*s2 + i3*s3]
struct Perm4 {
    const long long* offD; const long long* offS;
    int n0, n1, n2, n3;
    int d0, d1, d2, d3, s0, s1, s2, s3;
    int nbatch;
};
struct PermOp {
    double2* dst; const double2* src; const float2* src32; Perm4 p;
    __device__ void run(long long vb, long long nvb) const {
        const long long blk = (long long)p.n0 * p.n1 * p.n2 * p.n3;
        const long long total = blk * p.nbatch;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long b = e / blk;
            int r = (int)(e % blk);
            const int i3 = r % p.n3; r /= p.n3;
            const int i2 = r % p.n2; r /= p.n2;
            const int i1 = r % p.n1; const int i0 = r / p.n1;
            const long long so = p.offS[b] + (long long)i0 * p.s0 + (long long)i1 * p.s1 + (long long)i2 * p.s2 +
                                 (long long)i3 * p.s3;
            dst[p.offD[b] + (long long)i0 * p.d0 + (long long)i1 * p.d1 + (long long)i2 * p.d2 + (long long)i3 * p.d3] =
                src32 ? ldz(src32 + so) : ldz(src + so);
        }
    }
};
__global__ void permute4_kernel(const PermOp op) { op.run(blockIdx.x, gridDim.x); }

// R2 += Zr - Zr(i<->j) - Zr(a<->b) + Zr(both): the P_-(ij)P_-(ab) of Eq. ori_EqDouble
// (operator of Sec. 2; swapping an index swaps its momentum too).  The terms under
// P_-(ab) or P_-(ij) alone enter Zr at half weight (they are antisymmetric in the
// other index pair), so this one sum applies all three operators.
struct AntisymOp {
    double2* R2; const double2* Zr; const int* kb_of; int N, o, v;
    __device__ void run(long long vb, long long nvb) const {
        const long long blk = (long long)o * o * v * v;
        const long long total = (long long)N * N * N * blk;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long kk = e / blk;
            int r = (int)(e % blk);
            const int b = r % v; r /= v;
            const int a = r % v; r /= v;
            const int j = r % o; const int i = r / o;
            const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
            const int kb = kb_of[kk];
            // (ki,kj,ka)(i,j,a,b) ; (i<->j): (kj,ki,ka)(j,i,a,b) ; (a<->b): (ki,kj,kb)(i,j,b,a)
            const long long e_ij = (((long long)kj * N + ki) * N + ka) * blk + (((long long)j * o + i) * v + a) * v + b;
            const long long e_ab = (((long long)ki * N + kj) * N + kb) * blk + (((long long)i * o + j) * v + b) * v + a;
            const long long e_2 = (((long long)kj * N + ki) * N + kb) * blk + (((long long)j * o + i) * v + b) * v + a;
            const double2 z0 = Zr[e], z1 = Zr[e_ij], z2 = Zr[e_ab], z3 = Zr[e_2];
            double2 out = R2[e];
            out.x += z0.x - z1.x - z2.x + z3.x;
            out.y += z0.y - z1.y - z2.y + z3.y;
            R2[e] = out;
        }
    }
};
__global__ void antisym_kernel(const AntisymOp op) { op.run(blockIdx.x, gridDim.x); }

// Block-wise max |R| partials over an array (grid-stride; fixed per-thread order).
// part[vb] = max over this block's elements (blocks of 256 threads).
struct MaxabsOp {
    const double2* x; long long n; double* part;
    __device__ void run(long long vb, long long nvb) const {
        __shared__ double sm[256];
        double m = 0.0;
        for (long long e = vb * blockDim.x + threadIdx.x; e < n; e += nvb * blockDim.x) {
            const double2 z = x[e];
            const double a = sqrt(z.x * z.x + z.y * z.y);
            m = (a > m || a != a) ? a : m;     // NaN propagates
        }
        sm[threadIdx.x] = m;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double o2 = sm[threadIdx.x + s];
                if (o2 > sm[threadIdx.x] || o2 != o2) sm[threadIdx.x] = o2;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) part[vb] = sm[0];
    }
};
__global__ void maxabs_partial(const MaxabsOp op) { op.run(blockIdx.x, gridDim.x); }

// *out = max of n partials, in a fixed order (one thread of one block).
struct FinalMaxOp {
    const double* part; int n; double* out;
    __device__ void run(long long vb, long long) const {
        if (threadIdx.x == 0 && vb == 0) {
            double m = 0.0;
            for (int i = 0; i < n; ++i) { const double x = part[i]; if (x > m || x != x) m = x; }
            *out = m;
        }
    }
};

// t1 += R1 / D1, t2 += R2 / D2 (paper Sec. 4.4.19), D from the Fock diagonal
// eo[k][i], ev[k][a].  When err != nullptr also stores e = R / D (DIIS error).
struct UpdateOp {
    double2* t1; double2* t2;
    const double2* R1; const double2* R2;
    const double* eo; const double* ev;
    const int* kb_of; int N, o, v;
    double2* err1; double2* err2;
    const int* skip;          // batched form: a converged member (its flag set) is not updated
    __device__ void run(long long vb, long long nvb) const {
        if (skip && *skip) return;
        const long long n1 = (long long)N * o * v;
        const long long blk = (long long)o * o * v * v;
        const long long total = n1 + (long long)N * N * N * blk;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            if (e < n1) {
                const int a = (int)(e % v);
                const int i = (int)((e / v) % o);
                const int k = (int)(e / ((long long)o * v));
                const double d = eo[k * o + i] - ev[k * v + a];
                const double2 r = R1[e];
                const double2 q = make_double2(r.x / d, r.y / d);
                double2 t = t1[e];
                t.x += q.x; t.y += q.y;
                t1[e] = t;
                if (err1) err1[e] = q;
            } else {
                const long long f = e - n1;
                const long long kk = f / blk;
                int r = (int)(f % blk);
                const int b = r % v; r /= v;
                const int a = r % v; r /= v;
                const int j = r % o; const int i = r / o;
                const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
                const int kb = kb_of[kk];
                const double d = eo[ki * o + i] + eo[kj * o + j] - ev[ka * v + a] - ev[kb * v + b];
                const double2 rr = R2[f];
                const double2 q = make_double2(rr.x / d, rr.y / d);
                double2 t = t2[f];
                t.x += q.x; t.y += q.y;
                t2[f] = t;
                if (err2) err2[f] = q;
            }
        }
    }
};
__global__ void update_kernel(const UpdateOp op) { op.run(blockIdx.x, gridDim.x); }

// Energy partial sums: sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab
//                    + 1/2 sum_{ki,kj} <i ki j kj||a ki b kj> t_i^a t_j^b.
template <typename TS>
__global__ void energy_partial(const double2* __restrict__ t1, const double2* __restrict__ t2,
                               const double2* __restrict__ fov, const TS* __restrict__ oovv,
                               int N, int o, int v, double2* __restrict__ part)
{
    __shared__ double sr[256], si[256];
    const long long n1 = (long long)N * o * v;
    const long long blk = (long long)o * o * v * v;
    const long long n2 = (long long)N * N * N * blk;
    double er = 0.0, ei = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n1 + n2;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n1) {
            const double2 p = cmul(fov[e], t1[e]);
            er += p.x; ei += p.y;
        } else {
            const long long f = e - n1;
            const double2 g = ldz(oovv + f);
            double2 amp = t2[f];
            amp.x *= 0.25; amp.y *= 0.25;
            const long long kk = f / blk;
            const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
            if (ka == ki) {
                int r = (int)(f % blk);
                const int b = r % v; r /= v;
                const int a = r % v; r /= v;
                const int j = r % o; const int i = r / o;
                const double2 q = cmul(t1[((long long)ki * o + i) * v + a], t1[((long long)kj * o + j) * v + b]);
                amp.x += 0.5 * q.x; amp.y += 0.5 * q.y;
            }
            const double2 p = cmul(g, amp);
            er += p.x; ei += p.y;
        }
    }
    sr[threadIdx.x] = er; si[threadIdx.x] = ei;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sr[0], si[0]);
}

// Fixed-order final reductions (one block).
__global__ void final_max(const double* __restrict__ part, int n, double* __restrict__ out)
{
    FinalMaxOp{part, n, out}.run(blockIdx.x, gridDim.x);
}
__global__ void final_csum(const double2* __restrict__ part, int n, double2* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double r = 0.0, i2 = 0.0;
        for (int i = 0; i < n; ++i) { r += part[i].x; i2 += part[i].y; }
        *out = make_double2(r, i2);
    }
}

// ---------------------------------------------------------------------------
// Mixed form: the P(ab)-only and P(ij)-only terms of R2 at half weight, fused
// into one pass over Zr (FP32 products and sums, FP64 accumulation into Zr):
//   Zr += 1/2 sum_f t_ij^af F'^{bf}(kb) - 1/2 sum_r t_r^a(ka) <ij||rb>^*
//       - 1/2 sum_n t_in^ab F'_nj(kj)   - 1/2 sum_c t_i^c(ki) <jc||ab>^*
// (<ij||rb> = ooov[ki,kj,ka](i,j,r,b), <jc||ab> = ovvv[kj,ki,ka](j,c,a,b)); the
// same terms the FP64 form forms as four GEMMs.  Every short sum (o or v terms)
// is one thread's, so the pass reads t2 once and writes Zr once.
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfma_conjb(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// dst[k][c][r] = (complex64) src[k][r][c] for nk blocks of n x n
struct ToC64TOp {
    float2* dst; const double2* src; int nk, n;
    __device__ void run(long long vb, long long nvb) const {
        const long long total = (long long)nk * n * n;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long k = e / ((long long)n * n);
            const int rc = (int)(e % ((long long)n * n));
            const int c = rc / n, r = rc % n;
            const double2 z = src[(k * n + r) * n + c];
            dst[e] = make_float2((float)z.x, (float)z.y);
        }
    }
};
__global__ void to_c64_transpose_kernel(const ToC64TOp op) { op.run(blockIdx.x, gridDim.x); }

// fvvpT is F'^{bf} transposed per k: fvvpT[kb][f][b], so that the threads of a warp
// (consecutive b) read consecutive elements.
struct FockTermsOp {
    double2* Zr; const float2* t2; const float2* t1; const float2* fvvpT; const float2* foop;
    const float2* ooov; const float2* ovvv; const int* kb_of; int N, o, v;
    __device__ void run(long long vb, long long nvb) const {
        const long long blk = (long long)o * o * v * v;
        const long long total = (long long)N * N * N * blk;
        const long long vv = (long long)v * v, ov3 = (long long)o * v * vv, o3v = (long long)o * o * o * v;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            // thread order: b fastest, then i, a, j, the momentum block.  The o threads of
            // one (block, j, a, b) are neighbours, so their ovvv, F' and t1 reads (the
            // longest sum, over c) come from L1 after the first.
            long long w = e;
            const int b = (int)(w % v); w /= v;
            const int i = (int)(w % o); w /= o;
            const int a = (int)(w % v); w /= v;
            const int j = (int)(w % o);
            const long long kk = w / o;
            const long long eo = kk * blk + (((long long)i * o + j) * v + a) * v + b;   // Zr position
            const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
            const int kb = kb_of[kk];
            const float2* tb = t2 + kk * blk;
            float2 p = make_float2(0.f, 0.f), q = make_float2(0.f, 0.f);
            const float2* trow = tb + (((long long)i * o + j) * v + a) * v;             // t_ij^{a f}
            const float2* fcol = fvvpT + (long long)kb * v * v + b;                     // F'^{b f}(kb) at f v
#pragma unroll 4
            for (int f = 0; f < v; ++f) p = cfma(trow[f], fcol[(long long)f * v], p);
            const float2* oo = ooov + kk * o3v + ((long long)i * o + j) * o * v + b;    // <ij||r b>
            const float2* ta = t1 + (long long)ka * o * v + a;                          // t_r^a(ka)
#pragma unroll 4
            for (int rr = 0; rr < o; ++rr) q = cfma_conjb(ta[rr * v], oo[(long long)rr * v], q);
            const float2* tn = tb + ((long long)i * o * v + a) * v + b;                 // t_in^{ab}, n stride v^2
            const float2* fo = foop + (long long)kj * o * o + j;                        // F'_{n j}(kj)
#pragma unroll 4
            for (int n = 0; n < o; ++n) q = cfma(tn[(long long)n * vv], fo[n * o], q);
            const long long kjia = ((long long)kj * N + ki) * N + ka;
            const float2* vbp = ovvv + kjia * ov3 + (long long)j * v * vv + (long long)a * v + b;   // <j c||a b>
            const float2* ti = t1 + ((long long)ki * o + i) * v;                        // t_i^c(ki)
#pragma unroll 4
            for (int c = 0; c < v; ++c) q = cfma_conjb(ti[c], vbp[(long long)c * vv], q);
            double2 z = Zr[eo];
            z.x += 0.5 * ((double)p.x - (double)q.x);
            z.y += 0.5 * ((double)p.y - (double)q.y);
            Zr[eo] = z;
        }
    }
};
__global__ void fock_terms_kernel(const FockTermsOp op) { op.run(blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// Ozaki form: the same fused P(ab)-only / P(ij)-only terms in double-float arithmetic
// (about 48 bits, on the FP32 pipe), from double-float copies of t2, t1, F'vv
// (transposed per k), F'oo and ooov, and of ovvv (or complex64 integrals, which
// widen exactly):
//   Zr += 1/2 sum_f t_ij^af F'^{bf}(kb) - 1/2 sum_r t_r^a(ka) <ij||rb>^*
//       - 1/2 sum_n t_in^ab F'_nj(kj)   - 1/2 sum_c t_i^c(ki) <jc||ab>^*
// One thread per Zr element; the four short sums accumulate in double-float and
// Zr receives their FP64 sum.
__device__ __forceinline__ void cfma_df(const df2& a, const df2& b, df2& c) {
    c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
}
__device__ __forceinline__ void cfma_conjb_df(const df2& a, const df2& b, df2& c) {
    c.x = fma(a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
    c.y = fma(-a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
}
struct FockTermsDfOp {
    double2* Zr; const df2* t2; const df2* t1; const df2* fvvpT; const df2* foop;
    const df2* ooov; const float2* ooov32;       // double-float copy, or complex64 input
    const df2* ovvv; const float2* ovvv32;
    const int* kb_of; int N, o, v;
    __device__ void run(long long vb, long long nvb) const {
        const long long blk = (long long)o * o * v * v;
        const long long total = (long long)N * N * N * blk;
        const long long vv = (long long)v * v, ov3 = (long long)o * v * vv, o3v = (long long)o * o * o * v;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            const long long kk = e / blk;
            int r = (int)(e % blk);
            const int b = r % v; r /= v;
            const int a = r % v; r /= v;
            const int j = r % o; const int i = r / o;
            const int ka = (int)(kk % N), kj = (int)((kk / N) % N), ki = (int)(kk / ((long long)N * N));
            const int kb = kb_of[kk];
            const df2* tb = t2 + kk * blk;
            df2 p{df(0.f, 0.f), df(0.f, 0.f)}, q{df(0.f, 0.f), df(0.f, 0.f)};
            const df2* trow = tb + (((long long)i * o + j) * v + a) * v;              // t_ij^{a f}
            const df2* fcol = fvvpT + (long long)kb * v * v + b;                      // F'^{b f}(kb) at f v
            for (int f = 0; f < v; ++f) cfma_df(trow[f], fcol[(long long)f * v], p);
            const long long oo_off = kk * o3v + ((long long)i * o + j) * o * v + b;   // <ij||r b>
            const df2* ta = t1 + (long long)ka * o * v + a;                           // t_r^a(ka)
            for (int rr = 0; rr < o; ++rr) {
                const df2 w = ooov32 ? ld_df2(ooov32 + oo_off + (long long)rr * v) : ooov[oo_off + (long long)rr * v];
                cfma_conjb_df(ta[rr * v], w, q);
            }
            const df2* tn = tb + ((long long)i * o * v + a) * v + b;                  // t_in^{ab}, n stride v^2
            const df2* fo = foop + (long long)kj * o * o + j;                         // F'_{n j}(kj)
            for (int n = 0; n < o; ++n) cfma_df(tn[(long long)n * vv], fo[n * o], q);
            const long long kjia = ((long long)kj * N + ki) * N + ka;
            const long long vb_off = kjia * ov3 + (long long)j * v * vv + (long long)a * v + b;   // <j c||a b>
            const df2* ti = t1 + ((long long)ki * o + i) * v;                         // t_i^c(ki)
            for (int c = 0; c < v; ++c) {
                const df2 w = ovvv32 ? ld_df2(ovvv32 + vb_off + (long long)c * vv) : ovvv[vb_off + (long long)c * vv];
                cfma_conjb_df(ti[c], w, q);
            }
            const df2 d{p.x - q.x, p.y - q.y};
            double2 z = Zr[e];
            z.x += 0.5 * (double)d.x;
            z.y += 0.5 * (double)d.y;
            Zr[e] = z;
        }
    }
};
__global__ void fock_terms_df_kernel(const FockTermsDfOp op) { op.run(blockIdx.x, gridDim.x); }

// Double-float copies for fock_terms_df_kernel: t2 (n2 elements) into t2_df; t1 into
// t1_df, F'vv transposed per k into fvvpT_df, F'oo into foop_df.  Each element is split
// once (the split costs FP64 operations).
struct ToDfOp {
    df2* t2_df; const double2* t2; long long n2;
    df2* t1_df; const double2* t1; long long n1;
    df2* fvvpT_df; const double2* fvvp; df2* foop_df; const double2* foop; int N, o, v;
    __device__ void run(long long vb, long long nvb) const {
        const long long nv = (long long)N * v * v, no = (long long)N * o * o;
        const long long total = n2 + n1 + nv + no;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            if (e < n2) { t2_df[e] = ld_df2(t2 + e); continue; }
            long long f = e - n2;
            if (f < n1) { t1_df[f] = ld_df2(t1 + f); continue; }
            f -= n1;
            if (f < nv) {
                const long long k = f / ((long long)v * v);
                const int rc = (int)(f % ((long long)v * v));
                const int c = rc / v, r = rc % v;
                fvvpT_df[f] = ld_df2(fvvp + (k * v + r) * v + c);
                continue;
            }
            f -= nv;
            foop_df[f] = ld_df2(foop + f);
        }
    }
};
__global__ void to_df_kernel(const ToDfOp op) { op.run(blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// DIIS on the device (every handle, alone or in a group).  t2 is antisymmetric under
// (ki,i) <-> (kj,j) and under (ka,a) <-> (kb,b) (paper Sec. 2), so the blocks with
// ki <= kj and ka <= kb determine all others; a history vector holds t1 followed by
// those canonical blocks, and inner products weight each block by the number of
// full blocks it stands for.  An update packs x = t + R/D and e = R/D into history
// slot `next`, forms the weighted inner products of e with every filled slot, solves
// the Pulay system and writes x = sum c_h x_h to every block with the antisymmetry
// signs.  The history ring, the Gram matrix and the coefficients stay in device
// memory, so an iteration needs no host round trip and can be replayed from a graph.
struct DiisState {
    double2* hx[DIIS_MAX];    // history: amplitudes after the update (canonical blocks)
    double2* he[DIIS_MAX];    // history: errors R / D
    double gram[DIIS_MAX][DIIS_MAX];
    double coef[DIIS_MAX];
    int depth, next, count, m;
    int singular;             // a solve met a zero pivot (that iteration took the plain update)
};

// The reciprocal orbital-energy denominators 1 / D of the history's elements (t1,
// then the canonical t2 blocks; paper Sec. 4.4, Eqs. criterion_single and
// criterion_double), formed once at creation: an update then multiplies, where a
// division is a long sequence on the FP64 pipe (2 FMAs per clock and SM on GB300).
struct DiisRdenOp {
    double* rden; const int* cblk; long long nc;
    const double* eo; const double* ev; const int* kb_of; int N, o, v;
    __device__ void run(long long vb, long long nvb) const {
        const long long n1 = (long long)N * o * v;
        const long long blk = (long long)o * o * v * v;
        const long long total = n1 + nc * blk;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            double d;
            if (e < n1) {
                const int a = (int)(e % v);
                const int i = (int)((e / v) % o);
                const int k = (int)(e / ((long long)o * v));
                d = eo[k * o + i] - ev[k * v + a];
            } else {
                const long long pe = e - n1;
                const long long f = cblk[pe / blk];
                int r = (int)(pe % blk);
                const int b = r % v; r /= v;
                const int a = r % v; r /= v;
                const int j = r % o; const int i = r / o;
                const int ka = (int)(f % N), kj = (int)((f / N) % N), ki = (int)(f / ((long long)N * N));
                const int kb = kb_of[f];
                d = eo[ki * o + i] + eo[kj * o + j] - ev[ka * v + a] - ev[kb * v + b];
            }
            rden[e] = 1.0 / d;
        }
    }
};

// pack into slot ds->next, skipped for converged members: x = t + R / D, e = R / D on
// the canonical elements (R and t read at their full-array positions)
struct DiisPackOp {
    const double2* amp; const double2* res; DiisState* ds;
    const int* cblk; long long nc; const double* rden; int N, o, v;
    const int* skip;
    __device__ void run(long long vb, long long nvb) const {
        if (skip && *skip) return;
        const int slot = ds->next;
        double2* x_out = ds->hx[slot];
        double2* e_out = ds->he[slot];
        const long long n1 = (long long)N * o * v;
        const long long blk = (long long)o * o * v * v;
        const long long total = n1 + nc * blk;
        for (long long e = vb * blockDim.x + threadIdx.x; e < total; e += nvb * blockDim.x) {
            long long q = e;
            if (e >= n1) {
                const long long pe = e - n1;
                q = n1 + (long long)cblk[pe / blk] * blk + pe % blk;
            }
            const double rd = rden[e];
            const double2 rq = res[q];
            const double2 step = make_double2(rq.x * rd, rq.y * rd);
            const double2 t = amp[q];
            x_out[e] = make_double2(t.x + step.x, t.y + step.y);
            e_out[e] = step;
        }
    }
};

// Partial sums of w-weighted Re <e_next | e_j> for every slot j of the history
// (j >= the filled slots: zero).  Block r of nred takes the elements r * 256 + t
// (stride nred * 256) and forms all the slots' sums in one pass, so e_next is read
// once; part[j * nred + r] receives slot j's sum, each reduced over the block in the
// same fixed tree.
struct DiisDotOp {
    const DiisState* ds; long long n1, blk, nc; const double* cw;
    double* part; int nred;
    const int* skip;
    __device__ void run(long long vb, long long) const {
        if (skip && *skip) return;
        __shared__ double sm[256];
        const int r = (int)vb;
        const int m = min(ds->count + 1, ds->depth);
        const double2* x = ds->he[ds->next];
        const double2* y[DIIS_MAX];
#pragma unroll
        for (int j = 0; j < DIIS_MAX; ++j) y[j] = ds->he[j];
        double s[DIIS_MAX];
#pragma unroll
        for (int j = 0; j < DIIS_MAX; ++j) s[j] = 0.0;
        const long long n = n1 + nc * blk;
        for (long long e = (long long)r * blockDim.x + threadIdx.x; e < n; e += (long long)nred * blockDim.x) {
            const double2 a = x[e];
            const double w = e < n1 ? 1.0 : cw[(e - n1) / blk];
#pragma unroll
            for (int j = 0; j < DIIS_MAX; ++j) {
                if (j < m) {
                    const double2 b = y[j][e];
                    s[j] += w * (a.x * b.x + a.y * b.y);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < DIIS_MAX; ++j) {
            if (j >= ds->depth) break;
            sm[threadIdx.x] = s[j];
            __syncthreads();
            for (int st = blockDim.x / 2; st > 0; st >>= 1) {
                if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
                __syncthreads();
            }
            if (threadIdx.x == 0) part[j * nred + r] = sm[0];
            __syncthreads();
        }
    }
};

// One thread: the Gram row of the new slot (partials summed in a fixed order), the
// Pulay solve over the filled slots, and the ring advance.
struct DiisSolveOp {
    DiisState* ds; const double* part; int nred;
    const int* skip;
    __device__ void run(long long vb, long long) const {
        if ((skip && *skip) || vb != 0 || threadIdx.x >= 32) return;
        const int lane = threadIdx.x;
        const int slot = ds->next;
        const int m = min(ds->count + 1, ds->depth);
        // the partials of each slot: lane l sums r = l, l + 32, ... in order, then a fixed
        // shuffle tree over the lanes
        double g[DIIS_MAX];
#pragma unroll
        for (int j = 0; j < DIIS_MAX; ++j) {
            double d = 0.0;
            if (j < m)
                for (int r = lane; r < nred; r += 32) d += part[j * nred + r];
            for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xffffffffu, d, off);
            g[j] = d;
        }
        if (lane != 0) return;
        for (int j = 0; j < m; ++j) {
            ds->gram[slot][j] = g[j];
            ds->gram[j][slot] = g[j];
        }
        ds->count = m;
        ds->next = (slot + 1) % ds->depth;
        ds->m = m;
        for (int j = 0; j < DIIS_MAX; ++j) ds->coef[j] = 0.0;
        if (m < 2) { ds->coef[slot] = 1.0; return; }
        double c[DIIS_MAX];
        if (diis_solve(ds->gram, m, c)) {
            for (int j = 0; j < m; ++j) ds->coef[j] = c[j];
        } else {                  // singular: this iteration keeps the plain update
            ds->singular = 1;
            ds->coef[slot] = 1.0;
        }
    }
};

// amp = sum_h coef_h hx_h over the filled slots, written to every block.  The sum is
// formed once per canonical element and stored at each of the up to four full blocks
// the canonical block stands for (tgt[4 p + t] = 4 f + 2 swap_ij + swap_ab, -1 past the
// last), with the swapped indices and the antisymmetry sign.  Work units: t1 in pieces
// of 1024 elements, then 32 x 32 (a, b) tiles of every canonical (p, i, j) pair; a tile
// is staged in shared memory so that the (a, b)-swapped targets are written row by row
// as well (coalesced) instead of with a stride of v.
constexpr int DIIS_TILE = 32;
struct DiisComboOp {
    double2* out; const DiisState* ds; const int* tgt; long long nc; int N, o, v;
    const int* skip;
    __host__ __device__ long long units() const {
        const long long n1 = (long long)N * o * v;
        const long long nt = (v + DIIS_TILE - 1) / DIIS_TILE;
        return (n1 + 1023) / 1024 + nc * o * o * nt * nt;
    }
    __device__ void run(long long vb, long long nvb) const {
        if (skip && *skip) return;
        __shared__ double2 tile[DIIS_TILE][DIIS_TILE + 1];
        const int m = ds->m;
        const long long n1 = (long long)N * o * v;
        const long long blk = (long long)o * o * v * v;
        const long long u1 = (n1 + 1023) / 1024;
        const int nt = (v + DIIS_TILE - 1) / DIIS_TILE;
        const long long nu = u1 + nc * o * o * nt * nt;
        for (long long u = vb; u < nu; u += nvb) {
            if (u < u1) {                                   // t1: plain
                for (long long e = u * 1024 + threadIdx.x; e < min(n1, (u + 1) * 1024); e += blockDim.x) {
                    double re = 0.0, im = 0.0;
                    for (int h = 0; h < m; ++h) {
                        const double2 z = ds->hx[h][e];
                        re += ds->coef[h] * z.x;
                        im += ds->coef[h] * z.y;
                    }
                    out[e] = make_double2(re, im);
                }
                continue;
            }
            long long w = u - u1;
            const int tb = (int)(w % nt); w /= nt;
            const int ta = (int)(w % nt); w /= nt;
            const int j = (int)(w % o); w /= o;
            const int i = (int)(w % o);
            const long long p = w / o;
            const long long base = n1 + p * blk + ((long long)i * o + j) * v * v;   // canonical (i, j) plane
            for (int q = threadIdx.x; q < DIIS_TILE * DIIS_TILE; q += blockDim.x) {
                const int aa = q / DIIS_TILE, bb = q % DIIS_TILE;
                const int a = ta * DIIS_TILE + aa, b = tb * DIIS_TILE + bb;
                double re = 0.0, im = 0.0;
                if (a < v && b < v) {
                    const long long e = base + (long long)a * v + b;
                    for (int h = 0; h < m; ++h) {
                        const double2 z = ds->hx[h][e];
                        re += ds->coef[h] * z.x;
                        im += ds->coef[h] * z.y;
                    }
                }
                tile[aa][bb] = make_double2(re, im);
            }
            __syncthreads();
            for (int t = 0; t < 4; ++t) {
                const int g = tgt[4 * p + t];
                if (g < 0) break;
                const int sij = (g >> 1) & 1, sab = g & 1;
                const double sg = sij != sab ? -1.0 : 1.0;
                const long long fbase = n1 + (long long)(g >> 2) * blk +
                                        ((long long)(sij ? j : i) * o + (sij ? i : j)) * v * v;
                // target element (a2, b2) of the plane, b2 fastest; it holds canonical
                // (a, b) = (a2, b2), or (b2, a2) when the pair (a, b) is swapped
                const int a0 = sab ? tb : ta, b0 = sab ? ta : tb;
                for (int q = threadIdx.x; q < DIIS_TILE * DIIS_TILE; q += blockDim.x) {
                    const int x = q / DIIS_TILE, y = q % DIIS_TILE;
                    const int a2 = a0 * DIIS_TILE + x, b2 = b0 * DIIS_TILE + y;
                    if (a2 < v && b2 < v) {
                        const double2 z = sab ? tile[y][x] : tile[x][y];
                        out[fbase + (long long)a2 * v + b2] = make_double2(sg * z.x, sg * z.y);
                    }
                }
            }
            __syncthreads();
        }
    }
};

}  // namespace ccsdk
