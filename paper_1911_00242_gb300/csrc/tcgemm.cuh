// Tensor-core GEMM for the mixed form: tcgen05.mma kind::tf32, TMA-staged
// operands, FP32 accumulator in tensor memory (TMEM).
//
//   C'[m][n'] = sum_k A'[m][k] B'[n'][k]              (real, both K-major)
//
// A complex contraction C = A B^T becomes one real GEMM on the embedding
//   A'[m][2k + r] = (Re a_mk, Im a_mk)                 (= complex64 memory order)
//   B'[2n][2k + r] = (Re b_nk, -Im b_nk),  B'[2n+1][2k + r] = (Im b_nk, Re b_nk)
// so C'[m][2n] = Re c_mn and C'[m][2n+1] = Im c_mn (8 real flops per complex
// multiply-add, as 4M).  The split-TF32 option writes x = x_big + x_small with
// both parts TF32-exact and sums big*big + big*small + small*big, which keeps
// about 21 mantissa bits per product; the three terms are three passes over K
// into the same accumulator.
//
// Batch b and chunk c (a contracted momentum) select operand rows through
// tables: rows [rowA[b,c] + m0, +128) of the 2D TMA view of A', rows
// [rowB[b,c] + n0, +256) of B'.  The epilogue adds alpha * c_mn into an FP64
// result at offC[b*M + m] + colC[n].
//
// One CTA computes one 128 x 256 tile (cta_group::1, M = 128, N = 256):
//   warp 0 / lane 0 issues TMA loads into a 4-stage ring (48 KiB per stage),
//   warp 1 / lane 0 issues 4 MMAs (K = 8 each) per stage,
//   all 4 warps read the accumulator back with tcgen05.ld (warp w owns TMEM
//   lanes 32w..32w+31 = tile rows).
// Every mbarrier wait is bounded; on timeout the CTA records an error code,
// stops issuing, waits (bounded) for its copies in flight, frees its TMEM and
// returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccsdk {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 32;                                // fp32 elements per stage row (128 B)
constexpr int TC_STAGES = 4;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;            // 16 KiB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 4;            // 32 KiB
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;  // 48 KiB
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;
constexpr int TC_TMEM_COLS = 256;
constexpr long long TC_SPIN_LIMIT = 1LL << 24;           // polls before a wait gives up (> 0.1 s)
constexpr long long TC_DRAIN_LIMIT = 1LL << 20;          // polls per in-flight copy at teardown

struct TcArgs {
    const int* rowA;          // [nbatch * nchunk] row of A' where chunk c of batch b starts
    const int* rowB;          // [nbatch * nchunk]
    const long long* offC;    // [nbatch * M] complex-element offset of output row m
    const int* colC;          // [N/2] complex-element offset of output column n
    double2* C;               // FP64 result, C += alpha * c
    int* err;                 // error word (0 = ok)
    int M;                    // valid rows per batch
    int Nr;                   // valid real columns per batch (2 * complex columns)
    int nchunk;
    int kstages;              // K' / 32 per chunk
    int nterms;               // 1: A_big*B_big; 3: + A_big*B_small + A_small*B_big
    int tiles_m, tiles_n;
    double alpha_re, alpha_im;
    const int* nchunk_b;      // per-batch chunk count (<= nchunk) or null
    const long long* offC2;   // antisymmetric mirror: c is also subtracted at offC2[b*M+m] + colC2[n]
    const int* colC2;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase of parity `parity` to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit = TC_SPIN_LIMIT) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 1023) == 1023 && abort_flag && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar) : "memory");
}

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row atoms of
// 1024 bytes (stride byte offset 1024), leading byte offset unused (1).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);            // start address
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                   // stride byte offset
    d |= (uint64_t)1 << 46;                             // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                             // layout: SWIZZLE_128B
    return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 256, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

__global__ void __launch_bounds__(128, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA_big, const __grid_constant__ CUtensorMap mapA_small,
               const __grid_constant__ CUtensorMap mapB_big, const __grid_constant__ CUtensorMap mapB_small,
               const TcArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment for the swizzled stages
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stA = smem;                                        // [STAGES][16 KiB]
    uint8_t* stB = smem + TC_STAGES * TC_A_BYTES;               // [STAGES][32 KiB]
    uint64_t* bars = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars[0..S): full, bars[S..2S): empty, bars[2S]: accumulator ready
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * TC_STAGES + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntile = g.tiles_m * g.tiles_n;
    const int tile = blockIdx.x % ntile;
    const long long b = blockIdx.x / ntile;
    const int m0 = (tile % g.tiles_m) * TC_BM;
    const int n0 = (tile / g.tiles_m) * TC_BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[TC_STAGES + s]), 1);
        }
        mbar_init(smem_u32(&bars[2 * TC_STAGES]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32((const void*)tmem_slot)), "r"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int per_chunk = g.nterms * g.kstages;
    const int total = (g.nchunk_b ? g.nchunk_b[b] : g.nchunk) * per_chunk;
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // ---------------- producer: TMA loads
        for (int s = 0; s < total; ++s) {
            const int st = s % TC_STAGES;
            const uint32_t ph = (uint32_t)(s / TC_STAGES) & 1u;
            if (!mbar_wait(smem_u32(&bars[TC_STAGES + st]), ph ^ 1u, abort_flag)) {
                atomicCAS(g.err, 0, 1);
                *abort_flag = 1;
                break;
            }
            const int c = s / per_chunk;
            const int r = s % per_chunk;
            const int term = r / g.kstages;
            const int kx = (r % g.kstages) * TC_BK;
            const CUtensorMap* mA = (term == 2) ? &mapA_small : &mapA_big;
            const CUtensorMap* mB = (term == 1) ? &mapB_small : &mapB_big;
            const int ra = g.rowA[b * g.nchunk + c] + m0;
            const int rb = g.rowB[b * g.nchunk + c] + n0;
            const uint32_t full = smem_u32(&bars[st]);
            mbar_expect_tx(full, TC_STAGE_BYTES);
            tma_load_2d(smem_u32(stA + st * TC_A_BYTES), mA, kx, ra, full);
            tma_load_2d(smem_u32(stB + st * TC_B_BYTES), mB, kx, rb, full);
            issued = s + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = tc_idesc_tf32();
        bool ok = true;
        for (int s = 0; s < total; ++s) {
            const int st = s % TC_STAGES;
            const uint32_t ph = (uint32_t)(s / TC_STAGES) & 1u;
            if (!mbar_wait(smem_u32(&bars[st]), ph, abort_flag)) {
                atomicCAS(g.err, 0, 2);
                *abort_flag = 1;
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(stA + st * TC_A_BYTES);
            const uint32_t b0 = smem_u32(stB + st * TC_B_BYTES);
#pragma unroll
            for (int k = 0; k < TC_BK / 8; ++k) {           // K = 8 tf32 (32 bytes) per MMA
                tc_mma(tmem, smem_desc_sw128(a0 + 32 * k), smem_desc_sw128(b0 + 32 * k), idesc,
                       (s > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(smem_u32(&bars[TC_STAGES + st]));     // stage free once these MMAs have read it
        }
        if (ok) tc_commit(smem_u32(&bars[2 * TC_STAGES]));
        else {
            // nothing more will arrive on the accumulator barrier: release the epilogue
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&bars[2 * TC_STAGES])) : "memory");
        }
    }
    __syncwarp();

    // ---------------- epilogue: TMEM -> registers -> FP64 result
    bool acc_ok = mbar_wait(smem_u32(&bars[2 * TC_STAGES]), 0, nullptr) && !*abort_flag;
    acc_ok = __shfl_sync(0xffffffffu, acc_ok ? 1 : 0, 0) != 0;    // one decision per warp
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (acc_ok) {
        const int row = m0 + warp * 32 + lane;
        const bool rvalid = row < g.M;
        const long long rbase = rvalid ? g.offC[b * g.M + row] : 0;
        const long long rbase2 = (rvalid && g.offC2) ? g.offC2[b * g.M + row] : 0;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                           "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                           "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (rvalid) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int nr = n0 + c0 + 2 * q;                 // real column of the pair (re, im)
                    if (nr < g.Nr) {
                        const double xr = (double)__uint_as_float(v[2 * q]);
                        const double xi = (double)__uint_as_float(v[2 * q + 1]);
                        double2* p = g.C + rbase + g.colC[nr >> 1];
                        const double yr = g.alpha_re * xr - g.alpha_im * xi;
                        const double yi = g.alpha_re * xi + g.alpha_im * xr;
                        double2 o = *p;
                        o.x += yr; o.y += yi;
                        *p = o;
                        if (g.offC2) {
                            double2* q = g.C + rbase2 + g.colC2[nr >> 1];
                            double2 u = *q;
                            u.x -= yr; u.y -= yi;
                            *q = u;
                        }
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicCAS(g.err, 0, 3);
    }

    // ---------------- teardown: copies in flight, TMEM
    if (warp == 0 && lane == 0 && *abort_flag) {
        // wait (bounded) until every issued TMA has landed before the CTA exits
        for (int s = (issued > TC_STAGES ? issued - TC_STAGES : 0); s < issued; ++s)
            mbar_wait(smem_u32(&bars[s % TC_STAGES]), (uint32_t)(s / TC_STAGES) & 1u, nullptr, TC_DRAIN_LIMIT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------- operand prep
__device__ __forceinline__ float tf32_round(float x) {
    // round to nearest (ties away) at the 10-bit TF32 mantissa; TF32 MMAs then
    // use these values exactly
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    return __uint_as_float(u);
}

// Split of a float into TF32-exact big + small parts (FP32 arithmetic only).
__device__ __forceinline__ void split_tf32f(float x, float& big, float& small) {
    big = tf32_round(x);
    small = tf32_round(x - big);
}

// Split of a double into TF32-exact big + small parts.
__device__ __forceinline__ void split_tf32(double x, float& big, float& small) {
    const float f = (float)x;
    big = tf32_round(f);
    small = tf32_round((float)(x - (double)big));
}

}  // namespace ccsdk

namespace ccsdk {

// Operand preparation for tc_gemm_kernel: gathers a complex block matrix
// X_b[r][k] = src[srcoff[b] + srow[r] + scol[k]] and writes its real
// embedding, split into TF32-exact big and small parts:
//   mode 0 (A side): row b*R + r,           columns (2k, 2k+1) = (Re, Im)
//   mode 1 (B side): rows b*2R + 2r, +1,    columns (2k, 2k+1) = (Re, -Im) / (Im, Re)
// Row length Kpad >= 2 Kc; the padding columns are written as zero, so a buffer
// can be reused by operands of other shapes.
struct EmbedArgs {
    const double2* src; const float2* src32;   // source complex128, or complex64 when src32 is set
    const long long* srcoff; const int* srow; const int* scol;
    float* big; float* small;
    int nblk, R, Kc, Kpad, mode;
};

__global__ void embed_kernel(const EmbedArgs e)
{
    const int kh = e.Kpad / 2;                       // column pairs, padding included
    const long long total = (long long)e.nblk * e.R * kh;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(x % kh);
        const long long br = x / kh;
        const int r = (int)(br % e.R);
        const long long b = br / e.R;
        float rb = 0.f, rs = 0.f, ib = 0.f, is = 0.f;   // padding columns are written as zero
        if (k >= e.Kc) {
        } else if (e.src32) {
            const long long q = e.srcoff[b] + (long long)e.srow[r] + e.scol[k];
            const float2 z = e.src32[q];
            split_tf32f(z.x, rb, rs);
            split_tf32f(z.y, ib, is);
        } else {
            const long long q = e.srcoff[b] + (long long)e.srow[r] + e.scol[k];
            const double2 z = e.src[q];
            split_tf32(z.x, rb, rs);
            split_tf32(z.y, ib, is);
        }
        if (e.mode == 0) {
            const long long o = (b * e.R + r) * (long long)e.Kpad + 2LL * k;
            e.big[o] = rb; e.big[o + 1] = ib;
            if (e.small) { e.small[o] = rs; e.small[o + 1] = is; }
        } else {
            const long long o0 = (b * 2 * e.R + 2 * r) * (long long)e.Kpad + 2LL * k;
            const long long o1 = o0 + e.Kpad;
            e.big[o0] = rb; e.big[o0 + 1] = -ib;
            e.big[o1] = ib; e.big[o1 + 1] = rb;
            if (e.small) {
                e.small[o0] = rs; e.small[o0 + 1] = -is;
                e.small[o1] = is; e.small[o1 + 1] = rs;
            }
        }
    }
}

}  // namespace ccsdk

namespace ccsdk {

// dst = (complex64) src, n elements
__global__ void to_c64_kernel(float2* __restrict__ dst, const double2* __restrict__ src, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const double2 z = src[e];
        dst[e] = make_float2((float)z.x, (float)z.y);
    }
}

}  // namespace ccsdk

namespace ccsdk {

// Ladder operand W'^{abef} = <ab||ef> + sum_r t_r^b(kb) <r kb a ka||e ke f kf>
//                             - sum_r t_r^a(ka) <r ka b kb||e ke f kf>
// (the ovvv form of -P(ab) t_r^b <a r||e f>), formed in FP32 from complex64
// integrals and t1 and written straight into the B-side embedding of the
// antisymmetry-packed tensor-core ladder: output block bi is the momentum triple
// (ka, kb, ke) = blk[3 bi .. 3 bi + 2]; its rows are the listed (a, b) pairs
// (2 per pair) and its columns the listed (e, f) pairs:
// rows bi 2 nab + 2 ai + s, columns 2 ei + r; padding columns are written as zero.
struct WprimeListArgs {
    const float2* vvvv; const float2* ovvv; const float2* t1;
    float* big; float* small;
    const int* blk; const int* abl; const int* efl;
    int nblk, nab, nef, N, o, v, Kpad;
};

__global__ void wprime_list_kernel(const WprimeListArgs w)
{
    const int N = w.N, o = w.o, v = w.v;
    const long long vv = (long long)v * v, v4 = vv * vv, ov3 = (long long)o * v * vv;
    const int kh = w.Kpad / 2;                       // column pairs, padding included
    const long long per = (long long)w.nab * kh;
    const long long total = (long long)w.nblk * per;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const long long bi = x / per;
        const int r0 = (int)(x % per);
        const int ai = r0 / kh, ei = r0 % kh;
        const long long o0 = (bi * 2 * w.nab + 2LL * ai) * (long long)w.Kpad + 2LL * ei;
        const long long o1 = o0 + w.Kpad;
        if (ei >= w.nef) {                           // padding columns
            w.big[o0] = 0.f; w.big[o0 + 1] = 0.f; w.big[o1] = 0.f; w.big[o1 + 1] = 0.f;
            w.small[o0] = 0.f; w.small[o0 + 1] = 0.f; w.small[o1] = 0.f; w.small[o1 + 1] = 0.f;
            continue;
        }
        const int ka = w.blk[3 * bi], kb = w.blk[3 * bi + 1], ke = w.blk[3 * bi + 2];
        const int ab = w.abl[ai], ef = w.efl[ei];
        const int a = ab / v, b = ab % v;
        const long long blk_ab = ((long long)ka * N + kb) * N + ke;
        const long long blk_ba = ((long long)kb * N + ka) * N + ke;
        const float2 g = w.vvvv[blk_ab * v4 + (long long)ab * vv + ef];
        float sr = 0.f, si = 0.f;
        for (int r = 0; r < o; ++r) {
            const float2 tb = w.t1[((long long)kb * o + r) * v + b];
            const float2 p = w.ovvv[blk_ba * ov3 + ((long long)r * v + a) * vv + ef];
            sr = fmaf(tb.x, p.x, fmaf(-tb.y, p.y, sr));
            si = fmaf(tb.x, p.y, fmaf(tb.y, p.x, si));
            const float2 ta = w.t1[((long long)ka * o + r) * v + a];
            const float2 q = w.ovvv[blk_ab * ov3 + ((long long)r * v + b) * vv + ef];
            sr = fmaf(-ta.x, q.x, fmaf(ta.y, q.y, sr));
            si = fmaf(-ta.x, q.y, fmaf(-ta.y, q.x, si));
        }
        float rb, rs, ib, is;
        split_tf32f(g.x + sr, rb, rs);
        split_tf32f(g.y + si, ib, is);
        w.big[o0] = rb; w.big[o0 + 1] = -ib;
        w.big[o1] = ib; w.big[o1 + 1] = rb;
        w.small[o0] = rs; w.small[o0 + 1] = -is;
        w.small[o1] = is; w.small[o1 + 1] = rs;
    }
}

}  // namespace ccsdk
