// FP64-accurate complex contractions on the BF16 tensor cores (Ozaki scheme:
// Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59 (2012) 95-118).  The operands
// are split error-free into BF16 slices of small integers; the tensor core sums
// the slice products exactly, and the exact partial sums are added in a
// double-float register accumulator.
//
// Real embedding.  As for the split-TF32 kernel, a complex C = A B^T is the real
// GEMM C'[m][n'] = sum_k A'[m][k] B'[n'][k] with
//   A'[m][2k + r] = (Re a_mk, Im a_mk)
//   B'[2n][2k + r] = (Re b_nk, -Im b_nk),  B'[2n+1][2k + r] = (Im b_nk, Re b_nk).
//
// Splitting (per operand row).  Row i of an embedded operand gets a power-of-two
// scale 2^E_i > max_k |x_ik| and s slices of 7 bits: the fixed point
// Y = rint(x 2^{7s - E_i}) (|Y| <= 2^{7s}) is written in balanced base-128 digits,
// v_{s-1} .. v_1 in [-64, 63] from the least significant and the remaining top
// digit v_0 (|v_0| <= 128), so that
//   x = 2^E_i sum_{p<s} v_p 2^{-7(p+1)} + e,   |e| <= 2^{E_i - 7s - 1},
// with integers that BF16 holds exactly.
//
// Products.  With row scales 2^Ea (A') and 2^Eb (B'),
//   (A' B'^T)_mn = 2^{Ea_m + Eb_n} sum_{p,q} 2^{-7(p+q+2)} (V_p W_q^T)_mn.
// The pairs with p + q <= s - 1 are formed (s (s + 1) / 2 of them); the others
// lie below 2^{-7(s+1)} of 2^{Ea+Eb} per product.  Diagonal d = p + q has its own
// TMEM accumulator, which sums the products of all its pairs over one window of
// oz_kwin(s) K slices of one chunk; the window is short enough that every partial
// sum is an integer of magnitude <= 2^24, which FP32 holds exactly: the tensor-core
// accumulation is exact.  Each window sum is multiplied by its power of two (exact)
// and added into (hi, lo) with TwoSum (Knuth), so the only roundings after the
// split are those of the double-float sum.  The window factors are taken relative
// to the largest row scales of the output's chunks (RA for its A' rows, RB for its
// B' rows), so (hi, lo) stay near unit magnitude whatever the data's range; the
// epilogue multiplies by RA RB in FP64.
//
// One CTA computes a 128 x 64 tile (128 rows of A', 64 rows of B').  A stage is one
// K slice of 64: all s slices of the B tile (s x 8 KiB, in one of two B slots) and,
// one after another, the s slices of the A tile (16 KiB each, in a ring of A slots).
// Slice p of A meets slices q = 0 .. s-1-p of B, which lie side by side in the B slot,
// so one MMA of N = 64 n covers n consecutive q and writes the n adjacent diagonal
// accumulators p + q (TMEM columns 64 d).  Each staged byte thus feeds s / 2 products
// on average (one in a layout that stages one pair at a time), which keeps the shared
// memory's bandwidth, shared by the copies and the MMA operand reads, from bounding
// the tensor pipe.  Warp 0 / lane 0 issues the TMA loads, warp 1 / lane 0 the MMAs;
// warps 2..17 promote each diagonal's window as soon as its last product is in
// (diagonal p is complete once slice p of A is done in the window's last K slice) and
// keep (hi, lo) of 16 columns of one TMEM lane quarter in registers.  A launch with
// too few tiles for the SMs splits each tile's (chunk, window) units over several
// CTAs, whose partials oz_split_reduce adds in a fixed order.
// Every mbarrier wait is bounded, as in the split-TF32 kernel.
#pragma once
#include "tcgemm.cuh"
#include "dfloat.cuh"
#include "ozaki_split.cuh"
#include "ozaki_schedule.cuh"

namespace ccsdk {

constexpr int OZ_BM = 128;                                 // A' rows per tile (TMEM lanes)
constexpr int OZ_BN = 64;                                  // B' rows per tile (TMEM columns per diagonal)
constexpr int OZ_BK = 64;                                  // BF16 elements per K slice row (128 B)
static_assert(OZ_BK == 4 * 16, "the MMA issuer issues four K = 16 MMAs per K slice");
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;              // 16 KiB: one slice of the A tile
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;              // 8 KiB: one slice of the B tile
constexpr int OZ_RING_BYTES = 2 * OZ_MAX_SLICES * OZ_B_BYTES + 5 * OZ_A_BYTES;   // 208 KiB
constexpr int OZ_A_SLOTS = 12;                             // most A slots (s = 1); s = 7: 6
// A slices move in pairs of consecutive tiles of the load sequence (one full and one
// empty barrier per pair), which halves the issuer's waits and commits.
static_assert(OZ_MAX_SLICES * OZ_BN <= 512, "one TMEM accumulator per diagonal");
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_ACC_WARPS = 16;                           // four per TMEM lane quarter
constexpr int OZ_COLS = OZ_BN / (OZ_ACC_WARPS / 4);        // 16 columns per accumulator thread
static_assert(OZ_COLS % 8 == 0 && OZ_COLS <= 32, "columns per thread: 8-column TMEM loads, one lane each");
constexpr int OZ_THREADS = 64 + 32 * OZ_ACC_WARPS;
constexpr int OZ_MAX_SPLIT = 64;                           // most CTAs sharing one tile's units (small launches)
constexpr int OZ_BAR_BYTES = 512;                          // mbarriers, TMEM address, abort flag
constexpr int OZ_REF_BYTES = OZ_ACC_WARPS * 96 * 4;       // per accumulator warp: RB, 1 / RB, chunk column factors
constexpr int OZ_SMEM_BYTES = OZ_RING_BYTES + 1024 + OZ_BAR_BYTES + OZ_REF_BYTES;
static_assert((4 + OZ_A_SLOTS + 2 * OZ_MAX_SLICES + 1) * 8 + 8 <= OZ_BAR_BYTES, "barrier area");
static_assert(2 * OZ_COLS * (OZ_ACC_WARPS * 32) * 4 <= OZ_RING_BYTES, "epilogue park area");

struct OzArgs {
    const int* rowA;          // [nbatch * nchunk] row of A' (within a slice plane) where chunk c of batch b starts
    const int* rowB;          // [nbatch * nchunk]
    const long long* offC;    // [nbatch * M] complex-element offset of output row m (or [nbatch], rowC set)
    const int* rowC;          // null, or [M]: row m of batch b starts at offC[b] + rowC[m] (offC2 alike)
    const int* colC;          // [Nr / 2] complex-element offset of output column n
    double2* C;               // FP64 result, C += alpha * c
    int* err;                 // error word (0 = ok)
    const float* scA;         // [rowsA] row scales 2^E of A'
    const float* scB;         // [rowsB] row scales of B'
    int rowsA, rowsB;         // rows of one slice plane (plane p starts at row p * rows)
    int M, Nr, nchunk;
    int kstages;              // K' / 64 per chunk
    int slices;               // s (1 .. OZ_MAX_SLICES)
    int tiles_m, tiles_n;
    double alpha_re, alpha_im;
    const int* nchunk_b;      // per-batch chunk count (<= nchunk) or null
    const long long* offC2;   // antisymmetric mirror (subtracted) or null
    const int* colC2;
    long long spin_limit;
    int skip_stage;           // failure-detection self-test: this pair of A-slice loads is never issued (-1: none)
    int overwrite;            // 1: C = alpha c (and -alpha c at the mirror) instead of C += ...
    int nbatch;
    int nsplit;               // > 1: the (chunk, window) units of a tile are split over nsplit CTAs
    double2* work;            // nsplit > 1: partials [nsplit][nbatch][M][Nr / 2], summed by oz_split_reduce
};

// Instruction descriptor: D = F32, A = B = BF16 (kind::f16), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t oz_idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
}

// The four K = 16 steps (32 bytes each) of one 64-wide K slice into one accumulator:
// the first accumulates iff acc != 0, the others always.
__device__ __forceinline__ void oz_mma4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p, t;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "setp.eq.b32 t, %4, %4;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %6, %3, t;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %7, %8, %3, t;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %9, %10, %3, t;\n\t}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc), "l"(adesc + 2), "l"(bdesc + 2),
                    "l"(adesc + 4), "l"(bdesc + 4), "l"(adesc + 6), "l"(bdesc + 6) : "memory");
}

// 8 consecutive TMEM columns of this warp's lane quarter <-> registers (32x32b.x8).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                    "r"(r[7]) : "memory");
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// The MMAs of one K slice (the issuer of oz_gemm_kernel): for each A slice p (tile ja of
// the load sequence, half ja & 1 of pair slot ps; a pair is waited for at its first tile
// and released by one commit after its last), slices q0 .. q0+n-1 of B (adjacent in the
// B slot at descriptor dbs) in MMAs of N = 64 n into the accumulators of diagonals
// p + q0 .. (adjacent TMEM columns).  The first K step of p = 0 in a window's first K
// slice overwrites every diagonal, after the previous window's promotion of it; all
// later steps accumulate.  In the window's last K slice, diagonal p is complete after
// slice p of A, and its acc_full barrier is committed.  SC > 0: the slice count is a
// compile-time constant and the loops unroll; SC = 0: S at run time.  Returns 0, or the
// error code of a wait that gave up.
template <int SC>
__device__ __forceinline__ int oz_issue_slice(int S_rt, uint32_t tmem, uint64_t da0, uint64_t dbs, uint32_t fA0,
                                              uint32_t eA0, uint32_t accF0, uint32_t accE0, int nP, int totalA,
                                              int& ja, int& ps, uint32_t& pph, bool wfirst, bool wlast, int w,
                                              volatile int* abort_flag, long long spin_limit)
{
    const int S = SC > 0 ? SC : S_rt;
    const uint32_t id4 = oz_idesc_bf16(4 * OZ_BN);
#pragma unroll
    for (int p = 0; p < (SC > 0 ? SC : OZ_MAX_SLICES); ++p) {
        if (SC == 0 && p >= S) break;
        const int h = ja & 1;
        if (h == 0) {
            if (!mbar_wait(fA0 + 8 * ps, pph, abort_flag, spin_limit)) return 2;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const uint64_t da = da0 + (uint64_t)((2 * ps + h) * (OZ_A_BYTES >> 4));
        const bool fresh = wfirst && p == 0;
#pragma unroll
        for (int q0 = 0; q0 < (SC > 0 ? SC : OZ_MAX_SLICES); q0 += 4) {
            if (q0 >= S - p) break;
            const int n = min(4, S - p - q0);
            if (fresh && w > 0) {
                // diagonals q0 .. q0+n-1 of the previous window have been promoted
                for (int d = q0; d < q0 + n; ++d)
                    if (!mbar_wait(accE0 + 8 * d, (uint32_t)((w - 1) & 1), abort_flag, spin_limit)) return 4;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint64_t db = dbs + (uint64_t)(q0 * (OZ_B_BYTES >> 4));
            const uint32_t dst = tmem + (uint32_t)(OZ_BN * (p + q0));
            const uint32_t idesc = n == 4 ? id4 : oz_idesc_bf16(OZ_BN * n);
            oz_mma4(dst, da, db, idesc, fresh ? 0u : 1u);
        }
        if (h == 1 || ja + 1 == totalA) {
            tc_commit(eA0 + 8 * ps);
            if (++ps == nP) { ps = 0; pph ^= 1u; }
        }
        ++ja;
        if (wlast) tc_commit(accF0 + 8 * p);
    }
    return 0;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const OzArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int S = g.slices;
    const int bslot = S * OZ_B_BYTES;                           // all slices of one B tile
    const int nA = min(OZ_A_SLOTS, (OZ_RING_BYTES - 2 * bslot) / OZ_A_BYTES) & ~1;   // whole pairs
    uint8_t* stB = smem;                                        // [2][S][8 KiB]
    uint8_t* stA = smem + 2 * bslot;                            // [nA][16 KiB]
    const int nP = nA / 2;                                      // A pair slots
    uint64_t* fullB = (uint64_t*)(smem + OZ_RING_BYTES);
    uint64_t* emptyB = fullB + 2;
    uint64_t* fullA = fullB + 4;                                // per pair slot
    uint64_t* emptyA = fullA + OZ_A_SLOTS / 2;
    uint64_t* acc_full = emptyA + OZ_A_SLOTS / 2;               // per diagonal
    uint64_t* acc_empty = acc_full + OZ_MAX_SLICES;
    uint64_t* drain = acc_empty + OZ_MAX_SLICES;
    volatile uint32_t* tmem_slot = (volatile uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntile = g.tiles_m * g.tiles_n;
    const int tile = blockIdx.x % ntile;
    const long long b = (blockIdx.x / ntile) % g.nbatch;
    const int split = (int)(blockIdx.x / ntile / g.nbatch);
    const int m0 = (tile % g.tiles_m) * OZ_BM;
    const int n0 = (tile / g.tiles_m) * OZ_BN;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&fullB[i]), 1);
            mbar_init(smem_u32(&emptyB[i]), 1);
        }
        for (int i = 0; i < OZ_A_SLOTS / 2; ++i) {
            mbar_init(smem_u32(&fullA[i]), 1);
            mbar_init(smem_u32(&emptyA[i]), 1);
        }
        for (int d = 0; d < OZ_MAX_SLICES; ++d) {
            mbar_init(smem_u32(&acc_full[d]), 1);
            mbar_init(smem_u32(&acc_empty[d]), OZ_ACC_WARPS);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32((const void*)tmem_slot)), "r"(OZ_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int nch = g.nchunk_b ? g.nchunk_b[b] : g.nchunk;
    const int W = oz_kwin(S), nw = oz_nwin(g.kstages, S);
    int u0, u1;
    oz_unit_range(nch, S, g.kstages, g.nsplit, split, u0, u1);
    int nks = 0;                                                // K slices of this CTA
    for (int u = u0; u < u1; ++u) {
        const int k0 = (u % nw) * W;
        nks += min(k0 + W, g.kstages) - k0;
    }
    const int totalA = nks * S;                                 // A tiles of this CTA
    int issuedP = 0, issuedB = 0;                               // pairs / B slots loaded (warp 0 / lane 0)

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: per K slice, the B tile's S slices into B slot
            // (jb & 1), then the A tile's slices p = 0 .. S-1, pairs of consecutive tiles
            // (ja, ja + 1) into pair slot ps with one barrier.  Slot indices and phases
            // advance incrementally (no divisions in the loop).
            const uint32_t sA0 = smem_u32(stA), sB0 = smem_u32(stB);
            const uint32_t eA0 = smem_u32(&emptyA[0]), fA0 = smem_u32(&fullA[0]);
            int ja = 0, jb = 0, ps = 0;
            uint32_t pph = 0;
            bool skip = false, run = true;
            int open_x = 0, open_y = 0;                         // first tile of a half-loaded pair
            for (int u = u0; u < u1 && run; ++u) {
                const int c = u / nw, wi = u - c * nw;
                const int ra = g.rowA[b * g.nchunk + c] + m0, rb = g.rowB[b * g.nchunk + c] + n0;
                const int k1 = min((wi + 1) * W, g.kstages);
                for (int kst = wi * W; kst < k1 && run; ++kst) {
                    const int bs = jb & 1;
                    if (!mbar_wait(smem_u32(&emptyB[bs]), (uint32_t)((jb >> 1) & 1) ^ 1u, abort_flag, g.spin_limit)) {
                        run = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&fullB[bs]);
                    mbar_expect_tx(fb, (uint32_t)bslot);
                    for (int q = 0; q < S; ++q)
                        tma_load_2d(sB0 + bs * bslot + q * OZ_B_BYTES, &mapB, kst * OZ_BK, q * g.rowsB + rb, fb);
                    issuedB = ++jb;
                    for (int p = 0; p < S; ++p) {
                        const int h = ja & 1;
                        if (h == 0) {
                            if (!mbar_wait(eA0 + 8 * ps, pph ^ 1u, abort_flag, g.spin_limit)) {
                                run = false;
                                break;
                            }
                            skip = (ja >> 1) == g.skip_stage;  // a skipped pair is never loaded
                            if (!skip) {
                                mbar_expect_tx(fA0 + 8 * ps, (ja + 1 < totalA ? 2 : 1) * OZ_A_BYTES);
                                issuedP = (ja >> 1) + 1;
                            }
                            open_x = kst * OZ_BK;
                            open_y = p * g.rowsA + ra;
                        }
                        if (!skip)
                            tma_load_2d(sA0 + (2 * ps + h) * OZ_A_BYTES, &mapA, kst * OZ_BK, p * g.rowsA + ra, fA0 + 8 * ps);
                        ++ja;
                        if (h == 1 || ja == totalA) {
                            if (++ps == nP) { ps = 0; pph ^= 1u; }
                        }
                    }
                }
            }
            if (!run) {
                atomicCAS(g.err, 0, 1);
                *abort_flag = 1;
                // a pair left with one tile loaded gets its second load (the first tile again),
                // so that its barrier completes and teardown can wait for it
                if ((ja & 1) && ja < totalA && !skip)
                    tma_load_2d(sA0 + (2 * ps + 1) * OZ_A_BYTES, &mapA, open_x, open_y, fA0 + 8 * ps);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: per K slice, the B slot, then oz_issue_slice (the
            // slice count 7, the default, compiled as a constant).  The descriptors are the
            // slot-0 ones plus the slot offset (their start-address field is the shared
            // address / 16, below 2^14); slots and phases advance incrementally.
            const uint64_t da0 = smem_desc_sw128(smem_u32(stA)), db0 = smem_desc_sw128(smem_u32(stB));
            const uint32_t fA0 = smem_u32(&fullA[0]), eA0 = smem_u32(&emptyA[0]);
            const uint32_t accF0 = smem_u32(&acc_full[0]), accE0 = smem_u32(&acc_empty[0]);
            int ja = 0, ps = 0, bs = 0, w = 0;
            uint32_t pph = 0, bph = 0;
            int fail = 0;
            for (int u = u0; u < u1 && !fail; ++u, ++w) {
                const int k0 = (u % nw) * W, k1 = min(k0 + W, g.kstages);
                for (int kst = k0; kst < k1; ++kst) {
                    if (!mbar_wait(smem_u32(&fullB[bs]), bph, abort_flag, g.spin_limit)) {
                        fail = 2;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t dbs = db0 + (uint64_t)((bs * bslot) >> 4);
                    const bool wfirst = kst == k0, wlast = kst + 1 == k1;
                    fail = S == 7 ? oz_issue_slice<7>(S, tmem, da0, dbs, fA0, eA0, accF0, accE0, nP, totalA, ja, ps,
                                                      pph, wfirst, wlast, w, abort_flag, g.spin_limit)
                                  : oz_issue_slice<0>(S, tmem, da0, dbs, fA0, eA0, accF0, accE0, nP, totalA, ja, ps,
                                                      pph, wfirst, wlast, w, abort_flag, g.spin_limit);
                    if (fail) break;
                    tc_commit(smem_u32(&emptyB[bs]));
                    bs ^= 1;
                    if (bs == 0) bph ^= 1u;
                }
            }
            if (fail) {
                atomicCAS(g.err, 0, fail);
                *abort_flag = 1;
            }
            if (*abort_flag) {
                tc_commit(smem_u32(drain));
                mbar_wait(smem_u32(drain), 0u, nullptr, TC_DRAIN_LIMIT);
            }
        }
    } else {
        // ---------------- accumulator warps: exact window sums -> (hi, lo) in registers,
        // then the epilogue.  This thread: TMEM lane (row) 32 qr + lane, columns
        // cg * OZ_COLS .. + OZ_COLS of every diagonal.
        const int qr = warp & 3;
        const int cg = (warp - 2) >> 2;
        const int row = m0 + qr * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(qr * 32) << 16) + (uint32_t)(cg * OZ_COLS);
        float hi[OZ_COLS], lo[OZ_COLS];
#pragma unroll
        for (int i = 0; i < OZ_COLS; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
        // reference scales: RA over this row's chunks, RB over each column's (lane i: column i)
        float RA = 0.f, RBl = 0.f;
        const int col_l = n0 + cg * OZ_COLS + lane;
        const int c_lo = u0 / nw, c_hi = u1 > u0 ? (u1 - 1) / nw + 1 : c_lo;
        for (int c = c_lo; c < c_hi; ++c) {
            const int ra = g.rowA[b * g.nchunk + c] + row;
            if (row < g.M && ra < g.rowsA) RA = fmaxf(RA, g.scA[ra]);
            const int rb = g.rowB[b * g.nchunk + c] + col_l;
            if (lane < OZ_COLS && col_l < g.Nr && rb < g.rowsB) RBl = fmaxf(RBl, g.scB[rb]);
        }
        const float inv_ra = RA > 0.f ? 1.0f / RA : 0.f;        // exact: powers of two
        float* colref = (float*)(smem + OZ_RING_BYTES + OZ_BAR_BYTES) + (warp - 2) * 96;
        float* colfac = colref + 64;                            // this chunk's sb / RB per column
        colref[lane] = RBl;
        colref[32 + lane] = RBl > 0.f ? 1.0f / RBl : 0.f;
        __syncwarp();
        int cur_c = -1;
        bool ok = true;
        int w = 0;
        float sa = 0.f;
        for (int u = u0; u < u1 && ok; ++u, ++w) {
            const int c = u / nw;
            if (c != cur_c) {       // this row's factor; lane i: the factor of column i (one load each)
                const int ra = g.rowA[b * g.nchunk + c] + row;
                sa = (row < g.M && ra < g.rowsA) ? g.scA[ra] * inv_ra : 0.f;
                const int rbase = g.rowB[b * g.nchunk + c] + n0 + cg * OZ_COLS;
                const int nvalid = min(g.Nr - (n0 + cg * OZ_COLS), g.rowsB - rbase);
                __syncwarp();
                colfac[lane] = (lane < OZ_COLS && lane < nvalid) ? g.scB[rbase + lane] * colref[32 + lane] : 0.f;
                __syncwarp();
                cur_c = c;
            }
            for (int d = 0; d < S; ++d) {
                bool got = mbar_wait(smem_u32(&acc_full[d]), (uint32_t)(w & 1), abort_flag, g.spin_limit);
                got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                if (!got) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float fa = sa * __int_as_float((127 - OZ_SLICE_BITS * (d + 2)) << 23);  // * 2^{-7(d+2)}
#pragma unroll
                for (int c0 = 0; c0 < OZ_COLS; c0 += 8) {
                    uint32_t v[8];
                    tmem_ld8(tq + (uint32_t)(OZ_BN * d + c0), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        two_sum_acc(hi[c0 + i], lo[c0 + i], (__uint_as_float(v[i]) * colfac[c0 + i]) * fa);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acc_empty[d])) : "memory");
            }
        }
        if (ok && !*abort_flag) {
            if (row < g.M) {
                const long long rb0 = g.rowC ? g.offC[b] + g.rowC[row] : g.offC[b * g.M + row];
                const long long rb2 = !g.offC2 ? 0 : g.rowC ? g.offC2[b] + g.rowC[row] : g.offC2[b * g.M + row];
#pragma unroll
                for (int qq = 0; qq < OZ_COLS / 2; ++qq) {
                    const int nr = n0 + cg * OZ_COLS + 2 * qq;
                    if (nr >= g.Nr) continue;
                    const double xr = ((double)hi[2 * qq] + (double)lo[2 * qq]) * ((double)RA * (double)colref[2 * qq]);
                    const double xi = ((double)hi[2 * qq + 1] + (double)lo[2 * qq + 1]) *
                                      ((double)RA * (double)colref[2 * qq + 1]);
                    if (g.work) {       // partial of this split; oz_split_reduce applies alpha
                        g.work[(((long long)split * g.nbatch + b) * g.M + row) * (g.Nr / 2) + (nr >> 1)] =
                            make_double2(xr, xi);
                        continue;
                    }
                    const double yr = g.alpha_re * xr - g.alpha_im * xi;
                    const double yi = g.alpha_re * xi + g.alpha_im * xr;
                    double2* pc = g.C + rb0 + g.colC[nr >> 1];
                    double2 uu = g.overwrite ? make_double2(0.0, 0.0) : *pc;
                    uu.x += yr; uu.y += yi;
                    *pc = uu;
                    if (g.offC2) {
                        double2* p2 = g.C + rb2 + g.colC2[nr >> 1];
                        double2 z = g.overwrite ? make_double2(0.0, 0.0) : *p2;
                        z.x -= yr; z.y -= yi;
                        *p2 = z;
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
        for (int j = (issuedP > nP ? issuedP - nP : 0); j < issuedP; ++j)
            if (j != g.skip_stage)
                mbar_wait(smem_u32(&fullA[j % nP]), (uint32_t)(j / nP) & 1u, nullptr, TC_DRAIN_LIMIT);
        for (int j = (issuedB > 2 ? issuedB - 2 : 0); j < issuedB; ++j)
            mbar_wait(smem_u32(&fullB[j & 1]), (uint32_t)(j >> 1) & 1u, nullptr, TC_DRAIN_LIMIT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
    }
}

// Sum of the split partials in split order (deterministic), then the epilogue of
// oz_gemm_kernel: C (+)= alpha * sum at offC[b M + m] + colC[n] (and the mirror).
__global__ void oz_split_reduce(const OzArgs g)
{
    const int nc = g.Nr / 2;
    const long long n = (long long)g.nbatch * g.M * nc;
    const long long plane = n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        double xr = 0.0, xi = 0.0;
        for (int sp = 0; sp < g.nsplit; ++sp) {
            const double2 w = g.work[sp * plane + e];
            xr += w.x; xi += w.y;
        }
        const long long bm = e / nc;              // b * M + m
        const int col = (int)(e - bm * nc);
        const long long bb = bm / g.M;
        const int m = (int)(bm - bb * g.M);
        const double yr = g.alpha_re * xr - g.alpha_im * xi;
        const double yi = g.alpha_re * xi + g.alpha_im * xr;
        const long long r0 = g.rowC ? g.offC[bb] + g.rowC[m] : g.offC[bm];
        double2* p = g.C + r0 + g.colC[col];
        double2 u = g.overwrite ? make_double2(0.0, 0.0) : *p;
        u.x += yr; u.y += yi;
        *p = u;
        if (g.offC2) {
            double2* p2 = g.C + (g.rowC ? g.offC2[bb] + g.rowC[m] : g.offC2[bm]) + g.colC2[col];
            double2 z = g.overwrite ? make_double2(0.0, 0.0) : *p2;
            z.x -= yr; z.y -= yi;
            *p2 = z;
        }
    }
}

// ---------------------------------------------------------------- operand prep

__device__ __forceinline__ uint32_t pack_bf16x2(uint16_t lo, uint16_t hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long x, unsigned long long* red) {
    x = warp_max_u64(x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();                              // red[] of a previous row is no longer read
    if (lane == 0) red[warp] = x;
    __syncthreads();
    unsigned long long m = 0;
    for (int i = 0; i < nw; ++i) m = red[i] > m ? red[i] : m;
    return m;
}


// Operand preparation for oz_gemm_kernel (the Ozaki analogue of embed_kernel):
// gathers the complex block matrix X_b[r][k] = src[srcoff[b] + srow[r] + scol[k]],
// scales each embedded row by its power of two and writes the s slice planes:
//   mode 0 (A side): row b*R + r,         columns (2k, 2k+1) = (Re, Im)
//   mode 1 (B side): rows b*2R + 2r, +1,  columns (2k, 2k+1) = (Re, -Im) / (Im, Re)
// Plane p holds rows [0, rows) at sl + p * rows * Kpad; sc[row] = 2^E.
struct OzEmbedArgs {
    const double2* src; const float2* src32;
    const long long* srcoff; const int* srow; const int* scol;
    uint16_t* sl; float* sc;
    long long rows;           // rows of one plane
    int nblk, R, Kc, Kpad, mode, slices;
    int conj;                 // embed conj(X)
};

// One row (b, r), by a group of nthr threads (a warp or the CTA); tid is the thread's
// index in the group.  WARP: the group is one warp (no block barrier).
template <bool WARP, typename T>
__device__ __forceinline__ void oz_embed_row(const OzEmbedArgs& e, const T* src, long long br, int tid, int nthr,
                                             unsigned long long* red) {
    const int r = (int)(br % e.R);
    const long long b = br / e.R;
    const long long base = e.srcoff[b] + (long long)e.srow[r];
    unsigned long long m = 0;
    for (int k = tid; k < e.Kc; k += nthr) {
        const double2 z = ldz(src + base + e.scol[k]);
        const unsigned long long a = abs_bits(z.x), c = abs_bits(z.y);
        m = a > m ? a : m;
        m = c > m ? c : m;
    }
    m = WARP ? warp_max_u64(m) : block_max_u64(m, red);
    const int E = oz_row_exponent(m);
    const double fx = oz_fixed_scale(e.slices, E);
    const long long row0 = e.mode == 0 ? b * e.R + r : b * 2 * e.R + 2 * r;
    const long long plane = e.rows * (long long)e.Kpad;
    if (tid == 0) {
        e.sc[row0] = oz_row_scale(E);
        if (e.mode == 1) e.sc[row0 + 1] = oz_row_scale(E);
    }
    uint32_t* out0 = (uint32_t*)(e.sl + row0 * e.Kpad);
    const int kh = e.Kpad / 2;
    for (int k = tid; k < kh; k += nthr) {
        uint16_t sr[OZ_MAX_SLICES], si[OZ_MAX_SLICES];
        if (k < e.Kc) {
            const double2 z = ldz(src + base + e.scol[k]);
            oz_split(z.x, fx, e.slices, sr);
            oz_split(e.conj ? -z.y : z.y, fx, e.slices, si);
        } else {
            for (int p = 0; p < e.slices; ++p) { sr[p] = 0; si[p] = 0; }
        }
        for (int p = 0; p < e.slices; ++p) {
            uint32_t* o = out0 + (p * plane) / 2;
            if (e.mode == 0) {
                o[k] = pack_bf16x2(sr[p], si[p]);
            } else {
                o[k] = pack_bf16x2(sr[p], si[p] ^ 0x8000u);      // (Re, -Im)
                o[kh + k] = pack_bf16x2(si[p], sr[p]);           // (Im, Re)
            }
        }
    }
}

// Rows of at most 64 column pairs: one warp per row, 8 rows per CTA; longer rows: one
// CTA per row.
__global__ void oz_embed_kernel(const OzEmbedArgs e)
{
    __shared__ unsigned long long red[32];
    const long long rows = (long long)e.nblk * e.R;
    if (e.Kpad / 2 <= 64) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
        for (long long br = (long long)blockIdx.x * wpb + warp; br < rows; br += (long long)gridDim.x * wpb) {
            if (e.src32) oz_embed_row<true>(e, e.src32, br, lane, 32, red);
            else oz_embed_row<true>(e, e.src, br, lane, 32, red);
        }
        return;
    }
    for (long long br = blockIdx.x; br < rows; br += gridDim.x) {
        if (e.src32) oz_embed_row<false>(e, e.src32, br, threadIdx.x, blockDim.x, red);
        else oz_embed_row<false>(e, e.src, br, threadIdx.x, blockDim.x, red);
    }
}

// Ladder operand W'^{abef} (the same quantity as wprime_list_kernel forms in FP32),
// formed in FP64-class arithmetic (t1 terms in double-float, vvvv added in FP64) and
// written as Ozaki slices of the B-side embedding: output block
// bi is the momentum triple blk[3 bi ..], its rows the listed (a, b) pairs (2 per
// pair), its columns the listed (e, f) pairs; rows bi 2 nab + 2 ai + s.
struct OzWprimeArgs {
    const double2* vvvv; const float2* vvvv32;     // one of them
    const df2* ovvv_df; const float2* ovvv32;      // one of them (complex128 input: its double-float copy)
    const double2* t1;
    uint16_t* sl; float* sc;
    const int* blk; const int* abl; const int* efl;
    long long rows;           // rows of one plane
    int nblk, nab, nef, N, o, v, Kpad, slices;
};

// The t1 terms are summed in double-float (FP32 pipe) from a double-float copy of
// ovvv (or its complex64 values) and t1 values staged in shared memory.
template <typename TV, typename TO>
__device__ void oz_wprime_row(const OzWprimeArgs& w, const TV* vvvv, const TO* ovvv, long long row,
                              double2* vals, unsigned long long* red, df2* t1s) {
    const int N = w.N, o = w.o, v = w.v;
    const long long vv = (long long)v * v, v4 = vv * vv, ov3 = (long long)o * v * vv;
    const long long bi = row / w.nab;
    const int ai = (int)(row - bi * w.nab);
    const int ka = w.blk[3 * bi], kb = w.blk[3 * bi + 1], ke = w.blk[3 * bi + 2];
    const int ab = w.abl[ai];
    const int a = ab / v, b = ab % v;
    const long long blk_ab = ((long long)ka * N + kb) * N + ke;
    const long long blk_ba = ((long long)kb * N + ka) * N + ke;
    const TV* g0 = vvvv + blk_ab * v4 + (long long)ab * vv;
    const TO* pa = ovvv + blk_ba * ov3 + (long long)a * vv;         // + r v vv: ovvv[kb,ka,ke](r,a,.)
    const TO* pb = ovvv + blk_ab * ov3 + (long long)b * vv;         // ovvv[ka,kb,ke](r,b,.)
    // t1s[r] = t_r^b(kb), t1s[o + r] = -t_r^a(ka)
    __syncthreads();                              // t1s of the previous row is no longer read
    for (int r = threadIdx.x; r < 2 * o; r += blockDim.x) {
        if (r < o) {
            t1s[r] = ld_df2(w.t1 + (long long)kb * o * v + (long long)r * v + b);
        } else {
            const df2 z = ld_df2(w.t1 + (long long)ka * o * v + (long long)(r - o) * v + a);
            t1s[r] = df2{-z.x, -z.y};
        }
    }
    __syncthreads();
    unsigned long long m = 0;
    for (int ei = threadIdx.x; ei < w.nef; ei += blockDim.x) {
        const int ef = w.efl[ei];
        df2 s{df(0), df(0)};
        for (int r = 0; r < o; ++r) {
            // + t_r^b(kb) ovvv[kb,ka,ke](r,a,e,f) - t_r^a(ka) ovvv[ka,kb,ke](r,b,e,f)
            const df2 p = ld_df2(pa + (long long)r * v * vv + ef);
            const df2 tb = t1s[r];
            s.x = fma(tb.x, p.x, s.x); s.x = fma(-tb.y, p.y, s.x);
            s.y = fma(tb.x, p.y, s.y); s.y = fma(tb.y, p.x, s.y);
            const df2 q = ld_df2(pb + (long long)r * v * vv + ef);
            const df2 ta = t1s[o + r];
            s.x = fma(ta.x, q.x, s.x); s.x = fma(-ta.y, q.y, s.x);
            s.y = fma(ta.x, q.y, s.y); s.y = fma(ta.y, q.x, s.y);
        }
        double2 g = ldz(g0 + ef);
        g.x += (double)s.x;
        g.y += (double)s.y;
        vals[ei] = g;
        const unsigned long long a = abs_bits(g.x), c = abs_bits(g.y);
        m = a > m ? a : m;
        m = c > m ? c : m;
    }
    const int E = oz_row_exponent(block_max_u64(m, red));   // its barriers also publish vals[]
    const double fx = oz_fixed_scale(w.slices, E);
    const float scale = oz_row_scale(E);
    const long long row0 = bi * 2 * w.nab + 2LL * ai;
    const long long plane = w.rows * (long long)w.Kpad;
    if (threadIdx.x == 0) { w.sc[row0] = scale; w.sc[row0 + 1] = scale; }
    uint32_t* out0 = (uint32_t*)(w.sl + row0 * w.Kpad);
    const int kh = w.Kpad / 2;
    for (int k = threadIdx.x; k < kh; k += blockDim.x) {
        uint16_t sr[OZ_MAX_SLICES], si[OZ_MAX_SLICES];
        if (k < w.nef) {
            const double2 z = vals[k];
            oz_split(z.x, fx, w.slices, sr);
            oz_split(z.y, fx, w.slices, si);
        } else {
            for (int p = 0; p < w.slices; ++p) { sr[p] = 0; si[p] = 0; }
        }
        for (int p = 0; p < w.slices; ++p) {
            uint32_t* out = out0 + (p * plane) / 2;
            out[k] = pack_bf16x2(sr[p], si[p] ^ 0x8000u);
            out[kh + k] = pack_bf16x2(si[p], sr[p]);
        }
    }
    __syncthreads();                                  // vals[] is rewritten by the next row
}

// One CTA per output row pair; dynamic shared memory holds the row's nef values.
__global__ void oz_wprime_kernel(const OzWprimeArgs w)
{
    extern __shared__ double2 vals[];             // [nef] values, then [2 o] t1 values (df2)
    __shared__ unsigned long long red[32];
    df2* t1s = (df2*)(vals + w.nef);
    const long long rows = (long long)w.nblk * w.nab;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        if (w.vvvv32) {
            if (w.ovvv32) oz_wprime_row(w, w.vvvv32, w.ovvv32, row, vals, red, t1s);
            else oz_wprime_row(w, w.vvvv32, w.ovvv_df, row, vals, red, t1s);
        } else {
            if (w.ovvv32) oz_wprime_row(w, w.vvvv, w.ovvv32, row, vals, red, t1s);
            else oz_wprime_row(w, w.vvvv, w.ovvv_df, row, vals, red, t1s);
        }
    }
}

}  // namespace ccsdk
