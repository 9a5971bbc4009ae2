// Tensor-core GEMM for the mixed form: tcgen05.mma kind::tf32, TMA-staged
// operands, FP32 accumulators in tensor memory (TMEM).
//
//   C'[m][n'] = sum_k A'[m][k] B'[n'][k]              (real, both K-major)
//
// A complex contraction C = A B^T becomes one real GEMM on the embedding
//   A'[m][2k + r] = (Re a_mk, Im a_mk)                 (= complex64 memory order)
//   B'[2n][2k + r] = (Re b_nk, -Im b_nk),  B'[2n+1][2k + r] = (Im b_nk, Re b_nk)
// so C'[m][2n] = Re c_mn and C'[m][2n+1] = Im c_mn (8 real flops per complex
// multiply-add, as 4M).  The split-TF32 option writes x = x_big + x_small with
// both parts TF32-exact and sums big*big + big*small + small*big (each product
// to about 2^-22 relative); the three products of a K slice run on one staged copy
// of both parts.
//
// Accumulation.  The tensor core's FP32 accumulation truncates, so a long sum
// in one TMEM accumulator drifts by about half an ulp per MMA (1e-4 relative
// at K = 4096).  Every TC_PROMOTE_STAGES stages (18 MMAs) the partial is
// promoted: accumulator warps add it into FP32 registers (rounding to nearest)
// while the MMAs continue in the second TMEM accumulator.  Measured split-TF32
// error with promotion every 16 MMAs: 4e-7 .. 9e-7 of max|C| for K = 16 .. 4096.
//
// Batch b and chunk c (a contracted momentum) select operand rows through
// tables: rows [rowA[b,c] + m0, +128) of the 2D TMA view of A', rows
// [rowB[b,c] + n0, +256) of B'.  The epilogue adds alpha * c_mn into an FP64
// result at offC[b*M + m] + colC[n] (and subtracts it at the antisymmetric
// mirror offC2 / colC2 when given).
//
// One CTA computes one 128 x 256 tile (cta_group::1, M = 128, N = 256), 10 warps:
//   warp 0 / lane 0 issues TMA loads into a 4-stage ring (48 KiB per stage: a K
//   slice of 16 of both parts of A' and B', 64-byte swizzle),
//   warp 1 / lane 0 issues 6 MMAs (K = 8 each: two K steps of the three products)
//   per stage into TMEM buffer (segment & 1), warps 2..9 promote segments and run
//   the epilogue.
// Every mbarrier wait is bounded; on timeout the CTA records an error code,
// stops issuing, waits (bounded) for its copies and MMAs in flight, frees its
// TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tf32_split.cuh"

namespace ccsdk {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 16;                                // fp32 elements per stage row (64 B, 64-byte swizzle)
constexpr int TC_STAGES = 4;
static_assert((TC_STAGES & (TC_STAGES - 1)) == 0, "the ring index is s & (TC_STAGES - 1)");
static_assert(TC_BK == 2 * 8, "the MMA issuer issues two K = 8 MMAs per term and stage");
constexpr int TC_A_BYTES = TC_BM * TC_BK * 4;            // 8 KiB: one part (big or small) of the A tile
constexpr int TC_B_BYTES = TC_BN * TC_BK * 4;            // 16 KiB: one part of the B tile
// A stage holds both parts of both tiles, [A big | A small | B big | B small], so the
// three split-TF32 products of a K slice (big big, big small, small big) share one load:
// 6 MMAs per 48 KiB, where staging one term at a time needs 72 KiB for them.
constexpr int TC_STAGE_BYTES = 2 * (TC_A_BYTES + TC_B_BYTES);   // 48 KiB
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 + 256;
// Two TMEM accumulators of TC_BN columns: the MMAs fill one while the
// accumulator warps drain the other.
constexpr int TC_TMEM_COLS = 2 * TC_BN;
// Stages (6 MMAs of K = 8 each with split TF32) summed in TMEM before the partial is
// promoted into the FP32 register accumulator.  The tensor core's FP32 accumulation
// truncates: its error grows by about half an ulp of the running sum per MMA
// (measured with ccsd_tc_selftest: relative 2.6e-5 at K = 1024 complex, 1e-4 at
// K = 4096 with one TMEM sum per tile).  Promoting every 18 MMAs caps that bias
// at the partial of K = 48 reals per term; the register sums round to nearest.
constexpr int TC_PROMOTE_STAGES = 3;
constexpr int TC_ACC_WARPS = 8;                          // two per TMEM lane quarter, 128 columns each
constexpr int TC_THREADS = 64 + 32 * TC_ACC_WARPS;       // producer warp, MMA warp, accumulator warps
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
    long long spin_limit;     // polls before a wait gives up (TC_SPIN_LIMIT)
    int skip_stage;           // failure-detection self-test: this stage is never loaded (-1: none)
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
// The same for 64-byte swizzle: 8-row atoms of 512 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);            // start address
    d |= (uint64_t)1 << 16;                             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;                    // stride byte offset
    d |= (uint64_t)1 << 46;                             // descriptor version (tcgen05)
    d |= (uint64_t)4 << 61;                             // layout: SWIZZLE_64B
    return d;
}

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

// One 128 x 256 output tile of one batch: C[rows m][cols n] += alpha * sum over the
// batch's chunks, K stages and split terms of A'(rows) . B'(rows)^T.
//   warp 0, lane 0: TMA producer into a TC_STAGES ring (full/empty mbarriers)
//   warp 1, lane 0: MMA issuer; segment g of TC_PROMOTE_STAGES stages accumulates
//                   in TMEM buffer g & 1, then commits to acc_full[g & 1]
//   warps 2..9:     accumulator warps; warp w reads TMEM lanes 32 (w % 4) ..
//                   (its rows) and columns 128 ((w - 2) / 4) .. + 127 of each
//                   partial, adds them into FP32 registers, frees the buffer
//                   (acc_empty), and at the end adds alpha * sum into the FP64 C.
// Every wait is bounded; a timeout sets g.err and the CTA unwinds.
// `bid` is the CTA's tile index within its GEMM (tile + batch * tiles); the tensor maps
// sit in kernel-parameter space (one GEMM per launch) or in global memory (grouped
// launches of the batched form), written before the launch.
__device__ __forceinline__ void tc_gemm_body(const CUtensorMap* mapA_big, const CUtensorMap* mapA_small,
                                             const CUtensorMap* mapB_big, const CUtensorMap* mapB_small,
                                             const TcArgs& g, long long bid)
{
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment for the swizzled stages
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);
    // bars[0..S): full, bars[S..2S): empty, bars[2S + 0/1]: acc_full, bars[2S + 2/3]: acc_empty,
    // bars[2S + 4]: drain (abort path only)
    uint64_t* acc_full = bars + 2 * TC_STAGES;
    uint64_t* acc_empty = bars + 2 * TC_STAGES + 2;
    uint64_t* drain = bars + 2 * TC_STAGES + 4;
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(bars + 2 * TC_STAGES + 5);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntile = g.tiles_m * g.tiles_n;
    const int tile = (int)(bid % ntile);
    const long long b = bid / ntile;
    const int m0 = (tile % g.tiles_m) * TC_BM;
    const int n0 = (tile / g.tiles_m) * TC_BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[TC_STAGES + s]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&acc_full[i]), 1);
            mbar_init(smem_u32(&acc_empty[i]), TC_ACC_WARPS);
        }
        mbar_init(smem_u32(drain), 1);
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

    // one stage = one K slice of both parts of A and B; all terms of the slice run on it
    const bool split3 = g.nterms == 3;
    const int total = (g.nchunk_b ? g.nchunk_b[b] : g.nchunk) * g.kstages;
    const int nseg = (total + TC_PROMOTE_STAGES - 1) / TC_PROMOTE_STAGES;
    int issued = 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: TMA loads.  Chunk and K offset advance incrementally
            // (no divisions): this single thread's issue rate bounds the pipeline.
            const uint32_t s0 = smem_u32(smem);
            const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[TC_STAGES]);
            const uint32_t stage_tx = split3 ? TC_STAGE_BYTES : TC_A_BYTES + TC_B_BYTES;
            int c = 0, kx = 0;
            int ra = g.rowA[b * g.nchunk] + m0, rb = g.rowB[b * g.nchunk] + n0;
            for (int s = 0; s < total; ++s) {
                const int st = s & (TC_STAGES - 1);
                const uint32_t ph = (uint32_t)(s / TC_STAGES) & 1u;
                if (!mbar_wait(empty0 + 8 * st, ph ^ 1u, abort_flag, g.spin_limit)) {
                    atomicCAS(g.err, 0, 1);
                    *abort_flag = 1;
                    break;
                }
                if (s != g.skip_stage) {                   // a skipped stage is never completed
                    const uint32_t base = s0 + st * TC_STAGE_BYTES;
                    const uint32_t full = full0 + 8 * st;
                    mbar_expect_tx(full, stage_tx);
                    tma_load_2d(base, mapA_big, kx, ra, full);
                    tma_load_2d(base + 2 * TC_A_BYTES, mapB_big, kx, rb, full);
                    if (split3) {
                        tma_load_2d(base + TC_A_BYTES, mapA_small, kx, ra, full);
                        tma_load_2d(base + 2 * TC_A_BYTES + TC_B_BYTES, mapB_small, kx, rb, full);
                    }
                    issued = s + 1;
                }
                kx += TC_BK;
                if (kx == g.kstages * TC_BK) {
                    kx = 0;
                    if (++c < g.nchunk) {
                        ra = g.rowA[b * g.nchunk + c] + m0;
                        rb = g.rowB[b * g.nchunk + c] + n0;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer.  Stage descriptors: the stage-0 one plus the stage
            // and part offsets (the start-address field is the shared address / 16, below 2^14).
            const uint32_t idesc = tc_idesc_tf32();
            const uint64_t d0 = smem_desc_sw64(smem_u32(smem));
            const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[TC_STAGES]);
            for (int s = 0; s < total; ++s) {
                const int seg = s / TC_PROMOTE_STAGES;
                const int buf = seg & 1;
                const bool seg_first = (s % TC_PROMOTE_STAGES) == 0;
                if (seg_first && seg >= 2) {
                    // the accumulator warps must have drained this buffer's previous segment
                    if (!mbar_wait(smem_u32(&acc_empty[buf]), (uint32_t)((seg - 2) >> 1) & 1u, abort_flag, g.spin_limit)) {
                        atomicCAS(g.err, 0, 4);
                        *abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                const int st = s & (TC_STAGES - 1);
                const uint32_t ph = (uint32_t)(s / TC_STAGES) & 1u;
                if (!mbar_wait(full0 + 8 * st, ph, abort_flag, g.spin_limit)) {
                    atomicCAS(g.err, 0, 2);
                    *abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dab = d0 + (uint64_t)(st * (TC_STAGE_BYTES >> 4));   // A big
                const uint64_t das = dab + (uint64_t)(TC_A_BYTES >> 4);              // A small
                const uint64_t dbb = dab + (uint64_t)((2 * TC_A_BYTES) >> 4);        // B big
                const uint64_t dbs = dbb + (uint64_t)(TC_B_BYTES >> 4);              // B small
                const uint32_t dst = tmem + (uint32_t)(buf * TC_BN);
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {                                     // K = 8 tf32 (32 bytes) each
                    const uint64_t o = (uint64_t)(2 * kk);
                    tc_mma(dst, dab + o, dbb + o, idesc, (seg_first && kk == 0) ? 0u : 1u);
                    if (split3) {
                        tc_mma(dst, dab + o, dbs + o, idesc, 1u);
                        tc_mma(dst, das + o, dbb + o, idesc, 1u);
                    }
                }
                tc_commit(empty0 + 8 * st);                      // stage free once these MMAs have read it
                if ((s % TC_PROMOTE_STAGES) == TC_PROMOTE_STAGES - 1 || s == total - 1)
                    tc_commit(smem_u32(&acc_full[buf]));        // segment complete
            }
            if (*abort_flag) {
                // MMAs already issued must finish before the TMEM is released (bounded)
                tc_commit(smem_u32(drain));
                mbar_wait(smem_u32(drain), 0u, nullptr, TC_DRAIN_LIMIT);
            }
        }
    } else {
        // ---------------- accumulator warps: promote every segment, then the epilogue
        const int q = warp & 3;                                 // TMEM lane quarter = rows 32 q ..
        const int half = (warp - 2) >> 2;                       // columns 128 half ..
        float acc[TC_BN / 2];
#pragma unroll
        for (int i = 0; i < TC_BN / 2; ++i) acc[i] = 0.f;
        bool ok = true;
        for (int seg = 0; seg < nseg; ++seg) {
            const int buf = seg & 1;
            bool got = mbar_wait(smem_u32(&acc_full[buf]), (uint32_t)(seg >> 1) & 1u, abort_flag, g.spin_limit);
            got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;   // one decision per warp
            if (!got) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int c0 = 0; c0 < TC_BN / 2; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) +
                                       (uint32_t)(buf * TC_BN + half * (TC_BN / 2) + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                               "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c0 + i] += __uint_as_float(v[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acc_empty[buf])) : "memory");
        }
        if (ok && !*abort_flag) {
            // every MMA has completed (last acc_full), so the stage ring is free: park the
            // sums there to run the epilogue as a plain loop
            float* park = (float*)smem;                         // [TC_BN / 2][TC_ACC_WARPS * 32]
            const int t = (warp - 2) * 32 + lane;
#pragma unroll
            for (int i = 0; i < TC_BN / 2; ++i) park[i * (TC_ACC_WARPS * 32) + t] = acc[i];
            const int row = m0 + q * 32 + lane;
            if (row < g.M) {
                const long long rbase = g.offC[b * g.M + row];
                const long long rbase2 = g.offC2 ? g.offC2[b * g.M + row] : 0;
#pragma unroll 1
                for (int qq = 0; qq < TC_BN / 4; ++qq) {
                    const int nr = n0 + half * (TC_BN / 2) + 2 * qq;   // real column of the pair (re, im)
                    if (nr >= g.Nr) break;
                    const double xr = (double)park[(2 * qq) * (TC_ACC_WARPS * 32) + t];
                    const double xi = (double)park[(2 * qq + 1) * (TC_ACC_WARPS * 32) + t];
                    double2* p = g.C + rbase + g.colC[nr >> 1];
                    const double yr = g.alpha_re * xr - g.alpha_im * xi;
                    const double yi = g.alpha_re * xi + g.alpha_im * xr;
                    double2 o = *p;
                    o.x += yr; o.y += yi;
                    *p = o;
                    if (g.offC2) {
                        double2* p2 = g.C + rbase2 + g.colC2[nr >> 1];
                        double2 u = *p2;
                        u.x -= yr; u.y -= yi;
                        *p2 = u;
                    }
                }
            }
        } else if (lane == 0) {
            atomicCAS(g.err, 0, 3);
        }
    }

    // ---------------- teardown: copies in flight, TMEM
    __syncwarp();
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

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA_big, const __grid_constant__ CUtensorMap mapA_small,
               const __grid_constant__ CUtensorMap mapB_big, const __grid_constant__ CUtensorMap mapB_small,
               const TcArgs g)
{
    tc_gemm_body(&mapA_big, &mapA_small, &mapB_big, &mapB_small, g, blockIdx.x);
}

// Grouped form (batched form, serving rounds): one launch covers the same plan step of
// many independent problems.  CTA w works on member m with prefix[m] <= w < prefix[m+1],
// tile w - prefix[m] of that member's GEMM, with its arguments args[m] and its four
// tensor maps maps[4 m .. 4 m + 3] (A big, A small, B big, B small) from global memory.
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_grouped_kernel(const CUtensorMap* __restrict__ maps, const TcArgs* __restrict__ args,
                       const long long* __restrict__ prefix, int nmem)
{
    const long long w = blockIdx.x;
    int lo = 0, hi = nmem - 1;
    while (lo < hi) {                       // last member whose prefix <= w
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const TcArgs g = args[lo];
    const CUtensorMap* m = maps + 4 * lo;
    tc_gemm_body(m, m + 1, m + 2, m + 3, g, w - prefix[lo]);
}

}  // namespace ccsdk

namespace ccsdk {

// ---------------------------------------------------------------- operand prep
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
    // One block per operand row (b, r) of the (virtual) grid of nvb blocks: its threads
    // sweep the row's column pairs, so the per-element index arithmetic is one 32-bit add.
    __device__ void run(long long vb, long long nvb) const;
};

__device__ inline void EmbedArgs::run(long long vb, long long nvb) const
{
    const EmbedArgs& e = *this;
    const int kh = e.Kpad / 2;                       // column pairs, padding included
    const long long rows = (long long)e.nblk * e.R;
    for (long long br = vb; br < rows; br += nvb) {
        const int r = (int)(br % e.R);
        const long long b = br / e.R;
        const long long base = e.srcoff[b] + (long long)e.srow[r];
        const long long o = (e.mode == 0 ? (b * e.R + r) : (b * 2 * e.R + 2 * r)) * (long long)e.Kpad;
        for (int k = threadIdx.x; k < kh; k += blockDim.x) {
            float rb = 0.f, rs = 0.f, ib = 0.f, is = 0.f;   // padding columns are written as zero
            if (k < e.Kc) {
                const long long q = base + e.scol[k];
                if (e.src32) {
                    const float2 z = e.src32[q];
                    split_tf32f(z.x, rb, rs);
                    split_tf32f(z.y, ib, is);
                } else {
                    const double2 z = e.src[q];
                    split_tf32(z.x, rb, rs);
                    split_tf32(z.y, ib, is);
                }
            }
            const long long o0 = o + 2LL * k;
            if (e.mode == 0) {
                *(float2*)(e.big + o0) = make_float2(rb, ib);
                if (e.small) *(float2*)(e.small + o0) = make_float2(rs, is);
            } else {
                const long long o1 = o0 + e.Kpad;
                *(float2*)(e.big + o0) = make_float2(rb, -ib);
                *(float2*)(e.big + o1) = make_float2(ib, rb);
                if (e.small) {
                    *(float2*)(e.small + o0) = make_float2(rs, -is);
                    *(float2*)(e.small + o1) = make_float2(is, rs);
                }
            }
        }
    }
}

__global__ void embed_kernel(const EmbedArgs e) { e.run(blockIdx.x, gridDim.x); }

}  // namespace ccsdk

namespace ccsdk {

// dst = (complex64) src, n elements
struct ToC64Op {
    float2* dst; const double2* src; long long n;
    __device__ void run(long long vb, long long nvb) const {
        for (long long e = vb * blockDim.x + threadIdx.x; e < n; e += nvb * blockDim.x) {
            const double2 z = src[e];
            dst[e] = make_float2(f32_rn(z.x), f32_rn(z.y));    // integer rounding: no FP64 pipe
        }
    }
};
__global__ void to_c64_kernel(const ToC64Op op) { op.run(blockIdx.x, gridDim.x); }

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
    const int* grp;           // [ngrp][2]: first index into abl and count (<= WP_GROUP) of rows sharing a
    int nblk, nab, nef, N, o, v, Kpad, ngrp;
    __device__ void run(long long vb, long long nvb) const;
};

constexpr int WP_GROUP = 4;   // rows (pairs a b with one a) that share the ovvv row of a

// One CTA per group of up to WP_GROUP output row pairs of one block bi whose pairs (a, b)
// share a: the ovvv row of a and t_r^a are loaded once for the group, and its threads
// sweep the (e, f) list.
__device__ inline void WprimeListArgs::run(long long vb, long long nvb) const
{
    const WprimeListArgs& w = *this;
    const int N = w.N, o = w.o, v = w.v;
    const long long vv = (long long)v * v, v4 = vv * vv, ov3 = (long long)o * v * vv;
    const int kh = w.Kpad / 2;                       // column pairs, padding included
    const long long units = (long long)w.nblk * w.ngrp;
    for (long long unit = vb; unit < units; unit += nvb) {
        const long long bi = unit / w.ngrp;
        const int gi = (int)(unit - bi * w.ngrp);
        const int a0i = w.grp[2 * gi], cnt = w.grp[2 * gi + 1];
        const int ka = w.blk[3 * bi], kb = w.blk[3 * bi + 1], ke = w.blk[3 * bi + 2];
        const int a = w.abl[a0i] / v;
        const long long blk_ab = ((long long)ka * N + kb) * N + ke;
        const long long blk_ba = ((long long)kb * N + ka) * N + ke;
        const float2* pa = w.ovvv + blk_ba * ov3 + (long long)a * vv;     // + r v vv: ovvv[kb,ka,ke](r,a,.)
        const float2* ta = w.t1 + (long long)ka * o * v + a;              // t_r^a(ka)
        int bs[WP_GROUP];
#pragma unroll
        for (int g = 0; g < WP_GROUP; ++g) bs[g] = g < cnt ? w.abl[a0i + g] - a * v : 0;
        for (int ei = threadIdx.x; ei < kh; ei += blockDim.x) {
            if (ei >= w.nef) {                       // padding columns
                for (int g = 0; g < cnt; ++g) {
                    const long long o0 = (bi * 2 * w.nab + 2LL * (a0i + g)) * (long long)w.Kpad + 2LL * ei;
                    const long long o1 = o0 + w.Kpad;
                    *(float2*)(w.big + o0) = make_float2(0.f, 0.f);
                    *(float2*)(w.big + o1) = make_float2(0.f, 0.f);
                    *(float2*)(w.small + o0) = make_float2(0.f, 0.f);
                    *(float2*)(w.small + o1) = make_float2(0.f, 0.f);
                }
                continue;
            }
            const int ef = w.efl[ei];
            float sr[WP_GROUP], si[WP_GROUP];
#pragma unroll
            for (int g = 0; g < WP_GROUP; ++g) { sr[g] = 0.f; si[g] = 0.f; }
#pragma unroll 2
            for (int r = 0; r < o; ++r) {
                // + t_r^b(kb) ovvv[kb,ka,ke](r,a,e,f) - t_r^a(ka) ovvv[ka,kb,ke](r,b,e,f)
                const float2 p = pa[(long long)r * v * vv + ef];
                const float2 tar = ta[r * v];
#pragma unroll
                for (int g = 0; g < WP_GROUP; ++g) {
                    if (g >= cnt) break;
                    const float2 tbr = w.t1[(long long)kb * o * v + (long long)r * v + bs[g]];
                    const float2 q = w.ovvv[blk_ab * ov3 + (long long)bs[g] * vv + (long long)r * v * vv + ef];
                    sr[g] = fmaf(tbr.x, p.x, fmaf(-tbr.y, p.y, sr[g]));
                    si[g] = fmaf(tbr.x, p.y, fmaf(tbr.y, p.x, si[g]));
                    sr[g] = fmaf(-tar.x, q.x, fmaf(tar.y, q.y, sr[g]));
                    si[g] = fmaf(-tar.x, q.y, fmaf(-tar.y, q.x, si[g]));
                }
            }
#pragma unroll
            for (int g = 0; g < WP_GROUP; ++g) {
                if (g >= cnt) break;
                const int ab = a * v + bs[g];
                const float2 gv = w.vvvv[blk_ab * v4 + (long long)ab * vv + ef];
                float rb, rs, ib, is;
                split_tf32f(gv.x + sr[g], rb, rs);
                split_tf32f(gv.y + si[g], ib, is);
                const long long o0 = (bi * 2 * w.nab + 2LL * (a0i + g)) * (long long)w.Kpad + 2LL * ei;
                const long long o1 = o0 + w.Kpad;
                *(float2*)(w.big + o0) = make_float2(rb, -ib);
                *(float2*)(w.big + o1) = make_float2(ib, rb);
                *(float2*)(w.small + o0) = make_float2(rs, -is);
                *(float2*)(w.small + o1) = make_float2(is, rs);
            }
        }
    }
}

__global__ void wprime_list_kernel(const WprimeListArgs w) { w.run(blockIdx.x, gridDim.x); }

// The same W' rows, tiled for reuse: one unit is a tile of WPT_A consecutive a of one
// block and all their (a, b) pairs.  Per (e, f) column a thread keeps the ovvv rows of
// its a's (o values each) in registers and loads the ovvv row of every b once for the
// whole tile, where the grouped form above loads it once per (a, b) pair; t1 sits in
// shared memory.  Output rows are the pairs' positions in the list (all pairs, or
// a < b for the diagonal blocks ka = kb, both ordered by a then b).  o <= WPT_OMAX.
constexpr int WPT_A = 2;
constexpr int WPT_OMAX = 8;

struct WprimeTileOp {
    WprimeListArgs w;
    int lt;                   // the pair list holds a < b only (diagonal blocks)
    __device__ void run(long long vb, long long nvb) const {
        const int N = w.N, o = w.o, v = w.v;
        const long long vv = (long long)v * v, v4 = vv * vv, ov3 = (long long)o * v * vv;
        const int kh = w.Kpad / 2;
        const int ntile = (v + WPT_A - 1) / WPT_A;
        const long long units = (long long)w.nblk * ntile;
        __shared__ float2 tka[WPT_A * WPT_OMAX];                 // t_r^a(ka) of the tile's a
        __shared__ float2 tkb[WPT_OMAX * 128];                   // t_r^b(kb), b < 128
        for (long long unit = vb; unit < units; unit += nvb) {
            const long long bi = unit / ntile;
            const int a0 = (int)(unit - bi * ntile) * WPT_A;
            const int ka = w.blk[3 * bi], kb = w.blk[3 * bi + 1], ke = w.blk[3 * bi + 2];
            const long long blk_ab = ((long long)ka * N + kb) * N + ke;
            const long long blk_ba = ((long long)kb * N + ka) * N + ke;
            __syncthreads();                                       // the previous unit's reads are done
            // every entry the unrolled r loops read is written: r >= o reads as zero
            for (int q = threadIdx.x; q < WPT_A * WPT_OMAX; q += blockDim.x) {
                const int ta = q / WPT_OMAX, r = q % WPT_OMAX;
                tka[q] = (r < o && a0 + ta < v) ? w.t1[(long long)ka * o * v + (long long)r * v + a0 + ta]
                                                : make_float2(0.f, 0.f);
            }
            for (int q = threadIdx.x; q < WPT_OMAX * v; q += blockDim.x) {
                const int r = q % WPT_OMAX, b = q / WPT_OMAX;
                tkb[r * 128 + b] = r < o ? w.t1[(long long)kb * o * v + (long long)r * v + b] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            // first pair index of each a of the tile in the list
            int rowa[WPT_A];
#pragma unroll
            for (int ta = 0; ta < WPT_A; ++ta) {
                const int a = a0 + ta;
                rowa[ta] = lt ? a * v - a * (a + 1) / 2 - a - 1 : a * v;    // index of (a, b) = rowa + b
            }
            for (int ei = threadIdx.x; ei < kh; ei += blockDim.x) {
                if (ei >= w.nef) {                                 // padding columns of every row of the tile
                    for (int ta = 0; ta < WPT_A; ++ta) {
                        const int a = a0 + ta;
                        if (a >= v) break;
                        for (int b = lt ? a + 1 : 0; b < v; ++b) {
                            const long long o0 = (bi * 2 * w.nab + 2LL * (rowa[ta] + b)) * (long long)w.Kpad + 2LL * ei;
                            const long long o1 = o0 + w.Kpad;
                            *(float2*)(w.big + o0) = make_float2(0.f, 0.f);
                            *(float2*)(w.big + o1) = make_float2(0.f, 0.f);
                            *(float2*)(w.small + o0) = make_float2(0.f, 0.f);
                            *(float2*)(w.small + o1) = make_float2(0.f, 0.f);
                        }
                    }
                    continue;
                }
                const int ef = w.efl[ei];
                float2 P[WPT_A][WPT_OMAX];                         // ovvv[kb,ka,ke](r, a, ef)
#pragma unroll
                for (int ta = 0; ta < WPT_A; ++ta)
#pragma unroll
                    for (int r = 0; r < WPT_OMAX; ++r)
                        P[ta][r] = (r < o && a0 + ta < v)
                                       ? w.ovvv[blk_ba * ov3 + (long long)r * v * vv + (long long)(a0 + ta) * vv + ef]
                                       : make_float2(0.f, 0.f);
                for (int b = lt ? a0 + 1 : 0; b < v; ++b) {
                    float2 Q[WPT_OMAX];                            // ovvv[ka,kb,ke](r, b, ef)
#pragma unroll
                    for (int r = 0; r < WPT_OMAX; ++r)
                        Q[r] = r < o ? w.ovvv[blk_ab * ov3 + (long long)r * v * vv + (long long)b * vv + ef]
                                     : make_float2(0.f, 0.f);
#pragma unroll
                    for (int ta = 0; ta < WPT_A; ++ta) {
                        const int a = a0 + ta;
                        if (a >= v || (lt && a >= b)) continue;
                        // + t_r^b(kb) ovvv[kb,ka,ke](r,a,e,f) - t_r^a(ka) ovvv[ka,kb,ke](r,b,e,f)
                        float sr = 0.f, si = 0.f;
#pragma unroll
                        for (int r = 0; r < WPT_OMAX; ++r) {
                            const float2 tb = tkb[r * 128 + b], t_a = tka[ta * WPT_OMAX + r];
                            sr = fmaf(tb.x, P[ta][r].x, fmaf(-tb.y, P[ta][r].y, sr));
                            si = fmaf(tb.x, P[ta][r].y, fmaf(tb.y, P[ta][r].x, si));
                            sr = fmaf(-t_a.x, Q[r].x, fmaf(t_a.y, Q[r].y, sr));
                            si = fmaf(-t_a.x, Q[r].y, fmaf(-t_a.y, Q[r].x, si));
                        }
                        const float2 gv = w.vvvv[blk_ab * v4 + ((long long)a * v + b) * vv + ef];
                        float rb, rs, ib, is;
                        split_tf32f(gv.x + sr, rb, rs);
                        split_tf32f(gv.y + si, ib, is);
                        const long long o0 = (bi * 2 * w.nab + 2LL * (rowa[ta] + b)) * (long long)w.Kpad + 2LL * ei;
                        const long long o1 = o0 + w.Kpad;
                        *(float2*)(w.big + o0) = make_float2(rb, -ib);
                        *(float2*)(w.big + o1) = make_float2(ib, rb);
                        *(float2*)(w.small + o0) = make_float2(rs, -is);
                        *(float2*)(w.small + o1) = make_float2(is, rs);
                    }
                }
            }
        }
    }
};
__global__ void __launch_bounds__(256, 2) wprime_tile_kernel(const WprimeTileOp op) { op.run(blockIdx.x, gridDim.x); }


}  // namespace ccsdk
