// C ABI of the GB300 periodic-CCSD library: handle, plans, iteration driver.
//
// One residual evaluation is the sequence below (FP64 form).  Each
// contraction is one launch of the k-blocked complex GEMM (zgemm_kb.cuh); the
// batch index enumerates the two or three free momenta that the paper maps to
// process numbers (Sec. 3.1), the chunk index the contracted momentum that the
// paper's shifted SEND/RECV loop "Sum_88" walks (Sec. 4.3.4).
//
//   tau, tau~                                    Sec. 2 (tau definitions)
//   F~_ov, F~_oo, F~_vv                          Eqs. ori_F_ov, ori_F_oo, ori_F_vv
//   R1                                           Eq. ori_EqSingle
//   R2 = <ab||ij>
//      + 1/2 tau_mn^ab (W'_mnij + 1/2 X_mnij)    hole-hole: W~_mnij without its tau term
//                                                plus the 1/4 tau <mn||ef> part of W~^abef
//      + 1/2 tau_ij^ef W'^abef                   ladder: W~^abef without that part
//      + P(ij)P(ab) [t_in^af W~_jn^bf - t t <ov||vo>]   ring, Eq. Def_Woovv
//      + P(ab) F'vv t2 - P(ij) F'oo t2 + P(ij) <ab||cj> t - P(ab) t <rb||ij>
//   (X_mnij = sum tau_ij^ef <mn||ef>; both W~ factorizations are the
//    paper's Eq. ori_EqDouble regrouped, so R2 is unchanged)
// and the update t <- t + R/D with convergence test and energy (Sec. 4.4).
//
// The mixed and Ozaki forms add tensor-core variants of the ladder, ring and
// hole-hole contractions (steps of mode 2, tcgemm.cuh / ozaki.cuh) beside their FP64
// steps (mode 1); a handle runs one or the other per iteration.  The mixed form runs
// the remaining GEMMs in FP32 (and fuses the Fock terms), the Ozaki form runs them in
// double-float.
#include "../../include/ccsd.h"
#include "ccsd_kernels.cuh"
#include "tcgemm.cuh"
#include "ozaki.cuh"
#include "zgemm_kb.cuh"
#include "diis.h"
#include "grouped.cuh"
#include "kgrid.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

using namespace ccsdk;

namespace {

enum Buf {
    B_FOO_IN, B_FVV_IN, B_FOV_IN, B_OOOO, B_OOOV, B_OOVV, B_OVVO, B_OVVV, B_VVVV,
    B_T1, B_T2, B_R1, B_R2, B_TAU, B_TAUT,
    B_FOV, B_FOO, B_FVV, B_FOOP, B_FVVP,
    B_WHH, B_WAB, B_WRING, B_Q, B_TT, B_STA, B_STB, B_ZR,   // B_STA, B_STB: tensor-core self-test operands
    NBUF
};

struct GemmPlan {
    int a, b, c;
    GemmArgs args;      // device tables filled; A/B/C pointers resolved at launch
    GemmArgs args32;    // the same for the FP32 instance: shorter FP32 partial sums (split-K)
    int cfg;            // tile configuration
    int blocks;
};

struct CopyPlan {       // dst = (conj) src, n elements
    int dst, src; long long n; int conj;
};

struct PermPlan {
    int dst, src; Perm4 p;
};

struct Step {           // one element of the launch sequence
    int kind;           // 0 gemm, 1 copy, 2 perm, 3 tau, 4 antisym, 5 embed, 6 tensor-core gemm, 7 zero,
                        // 9 complex64 refresh of a buffer, 10 W' formation into the ladder's B operand,
                        // 11 fused Fock/t1 terms of R2 (mixed form), 12 transposed complex64 F'vv
    int idx;
    const char* name;
    double flops;       // algorithmic real flops per launch (complex MAC = 8)
    double bytes;       // algorithmic bytes per launch for the memory-bound steps
    int mode = 0;       // 0 always; 1 only without tensor cores; 2 split-TF32 tensor-core steps
                        // (mixed iterations); 3 only in mixed iterations; 4 only outside them;
                        // 5 Ozaki tensor-core steps (Ozaki iterations)
};

struct EmbedPlan {      // operand preparation for the tensor-core GEMM
    int src;
    bool oz = false;    // Ozaki slices (z) instead of split-TF32 parts (a)
    EmbedArgs a;        // a.src resolved at launch
    OzEmbedArgs z;
};

struct WListPlan {      // fused W' formation + embedding for listed blocks and index pairs
    bool oz = false;
    WprimeListArgs a;
    OzWprimeArgs z;
};

struct TcPlan {
    CUtensorMap mA_big, mA_small, mB_big, mB_small;   // Ozaki: mA_big / mB_big map the slice planes
    bool oz = false;
    TcArgs a;           // a.C resolved at launch
    OzArgs z;
    int c;
    int blocks;
};

}  // namespace

struct ccsd_ctx {
    ccsd_config cfg;
    KGrid kg;
    int N = 0, o = 0, v = 0;
    long long n1 = 0, n2 = 0;       // elements of t1 and t2
    cudaStream_t st = nullptr;
    double2* buf[NBUF] = {};
    long long bufsize[NBUF] = {};   // elements, for plan bound checks
    float2* shadow[NBUF] = {};       // complex64 data: mixed-form copies, or inputs stored complex64
    bool in32[NBUF] = {};            // input stored complex64 only (shadow[] set, buf[] null)
    std::vector<void*> owned;        // device allocations to free
    void* host_registered = nullptr; // host vvvv registered (or counted) by the library; released at destroy
    size_t owned_bytes = 0;
    double2* amp = nullptr;          // [t1 | t2]
    double2* res = nullptr;          // [R1 | R2]
    double* eo = nullptr;            // Fock diagonal eo[k][i]
    double* ev = nullptr;            // ev[k][a]
    int* kb_of = nullptr;            // fourth momentum of doubles blocks
    double2* work = nullptr;         // split-K partials
    size_t work_elems = 0;
    double* red = nullptr;           // reduction partials
    double* red_out = nullptr;       // scalars
    double2* cred = nullptr;
    double2* cred_out = nullptr;
    double* norm_host = nullptr;     // pinned: max|R| of the last iteration
    cudaEvent_t ev_norm = nullptr;
    std::vector<double2*> hx, he;    // DIIS history on canonical blocks: [t1 | nc blocks of t2]
    long long nc = 0;                // canonical t2 blocks (ki <= kj, ka <= kb)
    int* d_cblk = nullptr;           // full block index of each canonical block
    double* d_cw = nullptr;          // its weight: the number of blocks it stands for
    double* d_rden = nullptr;        // 1 / D of the history's elements (t1, canonical t2 blocks)
    int* d_ctgt = nullptr;           // per canonical block: up to 4 full blocks it stands for,
                                     // 4 * full index + 2 swap_ij + swap_ab (-1 past the last)
    DiisState* d_diis = nullptr;     // DIIS state on the device (history ring, Gram matrix, coefficients)
    double* d_diis_part = nullptr;   // [depth][red_blocks] inner-product partials
    DiisState diis_init{};           // its initial value (empty history), for resets
    std::vector<GemmPlan> gemms;
    std::vector<CopyPlan> copies;
    std::vector<PermPlan> perms;
    std::vector<Step> seq;
    long long launches = 0;
    int red_blocks = 0;
    const char* cur_name = "";
    int fp32 = 0;                    // contractions in FP32 arithmetic (mixed form)
    int oz_on = 0;                   // Ozaki-scheme tensor-core contractions active this iteration
    bool has_oz = false;             // the plan has the Ozaki steps (CCSD_OZAKI, or the mixed form's Ozaki polish)
    bool cur_oz = false;             // plan building: the operand set being added is the Ozaki one
    int oz_slices = 7;               // slices per operand row (CCSD_OZAKI)
    long long oz_work_elems = 0;     // split partials of the Ozaki GEMMs (complex elements)
    df2* ovvv_df = nullptr;          // Ozaki form, complex128 ovvv: its double-float copy
    df2* ooov_df = nullptr;          // the same for complex128 ooov (fused Fock terms)
    df2* t2_df = nullptr;            // Ozaki iterations: double-float copies for the fused Fock
    df2* t1_df = nullptr;            // terms (t2_df aliases the idle B operand pool in the
    df2* fvvpT_df = nullptr;         // pooled layout)
    df2* foop_df = nullptr;
    double2* oz_work = nullptr;
    long long wab_cap_bytes = 12LL << 30;   // bound of the ladder's W' slab buffer
    // mixed and Ozaki forms: tensor-core operands (TF32 big/small parts, or BF16 slice
    // planes and row scales, of the real embeddings)
    std::vector<EmbedPlan> embeds;
    std::vector<TcPlan> tcs;
    std::vector<WListPlan> wlists;
    std::vector<int> const_embeds;   // embeds of constant inputs, run once at creation
    int* tc_err = nullptr;
    // tracing: CUDA events around every step of the residual plan
    int trace = 0;
    std::vector<cudaEvent_t> ev0, ev1;
    std::vector<double> step_ms;
    std::vector<long long> step_calls;
};

namespace {

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { last_err(e_); return CCSD_ERR_CUDA; } } while (0)
thread_local char g_errbuf[256];
void last_err(cudaError_t e) { snprintf(g_errbuf, sizeof g_errbuf, "%s", cudaGetErrorString(e)); }

// Records why a configuration or a call is refused (ccsd_last_error).
bool refuse(const char* why) {
    snprintf(g_errbuf, sizeof g_errbuf, "%s", why);
    return false;
}

// Every exported entry point opens one: the outermost call on a thread clears the
// message of ccsd_last_error, calls nested inside it (a failed create destroying its
// handle, a solve resetting the precision) keep what the failure recorded.
thread_local int g_api_depth = 0;
struct ApiScope {
    ApiScope() { if (g_api_depth++ == 0) g_errbuf[0] = 0; }
    ~ApiScope() { --g_api_depth; }
    ApiScope(const ApiScope&) = delete;
    ApiScope& operator=(const ApiScope&) = delete;
};

struct Alloc {
    ccsd_ctx* h;
    int err = 0;
    bool dry = false;     // plan validation only: no device memory, no copies
    void* get(size_t bytes) {
        if (err) return nullptr;
        void* p = nullptr;
        if (bytes == 0) bytes = 16;
        if (dry) { h->owned_bytes += bytes; return (void*)(uintptr_t)256; }
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); err = (e == cudaErrorMemoryAllocation) ? CCSD_ERR_OOM : CCSD_ERR_CUDA; return nullptr; }
        h->owned.push_back(p);
        h->owned_bytes += bytes;
        return p;
    }
};

template <class T>
T* upload(Alloc& al, const std::vector<T>& v, cudaStream_t st) {
    T* d = (T*)al.get(v.size() * sizeof(T));
    if (!d) return nullptr;
    if (al.dry) return d;
    if (cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess) { al.err = CCSD_ERR_CUDA; return nullptr; }
    if (cudaStreamSynchronize(st) != cudaSuccess) { al.err = CCSD_ERR_CUDA; return nullptr; }
    return d;
}

// Table helpers: idx(x) for x over a product of index ranges with strides.
std::vector<int> tab(std::initializer_list<std::pair<int, long long>> dims) {
    std::vector<std::pair<int, long long>> d(dims);
    long long total = 1;
    for (auto& p : d) total *= p.first;
    std::vector<int> out((size_t)total);
    for (long long x = 0; x < total; ++x) {
        long long r = x, off = 0;
        for (int i = (int)d.size() - 1; i >= 0; --i) { off += (r % d[i].first) * d[i].second; r /= d[i].first; }
        out[(size_t)x] = (int)off;
    }
    return out;
}

struct GemmSpec {
    int a, b, c;
    int M, N, K, nbatch, nchunk;
    std::vector<long long> offA, offB, offC;
    std::vector<int> rowA, colA, rowB, colB, rowC, colC;
    std::vector<int> nchunk_b;               // optional per-batch chunk counts
    std::vector<long long> offC2;            // optional antisymmetric mirror of C
    std::vector<int> colC2;
    bool conjA = false, conjB = false, acc = true;
    double ar = 1.0, ai = 0.0;
};

// Tile configurations: (BM, BN, BK, TM, TN[, KS]), 256 threads each.  The two K-split
// shapes (KS thread groups share each K step) serve skinny contractions with K >= 32.
enum { CFG_64x64 = 0, CFG_64x32 = 1, CFG_128x16 = 2, CFG_16x16 = 3, CFG_32x16 = 4, CFG_16x16K = 5, CFG_32x16K = 6,
       CFG_COUNT = 7 };
const int CFG_BM[CFG_COUNT] = {64, 64, 128, 16, 32, 16, 32};
const int CFG_BN[CFG_COUNT] = {64, 32, 16, 16, 16, 16, 16};

const int kSMs = 152;
const int kRedBlocks = kSMs * 4;    // blocks of the reductions (max|R|, inner products, energy)

// Momentum pairs (ka <= kb) whose ladder W' blocks one slab holds: as many as fit in
// cap bytes, at least one.  The slab buffer holds that many pairs x N blocks of v^4.
long long wab_pairs_per_slab(long long N, long long v, long long cap) {
    const long long pairs = N * (N + 1) / 2;
    const long long pair_bytes = 16 * N * v * v * v * v;
    return std::max<long long>(1, std::min<long long>(pairs, cap / pair_bytes));
}

int finalize_gemm(ccsd_ctx* h, Alloc& al, GemmSpec s, size_t& work_need) {
    if (s.nbatch == 0) {
        // an empty contraction (no momentum blocks for this shape): kept as a no-op step
        // so that every problem has the same step sequence (batched form)
        GemmPlan p{};
        p.a = s.a; p.b = s.b; p.c = s.c; p.cfg = CFG_16x16; p.blocks = 0;
        p.args.M = std::max(s.M, 1); p.args.N = std::max(s.N, 1); p.args.K = s.K;
        p.args.nbatch = 0; p.args.nchunk = std::max(s.nchunk, 1); p.args.nsplit = 1; p.args.chunks_per_split = 1;
        h->gemms.push_back(p);
        h->seq.push_back({0, (int)h->gemms.size() - 1, h->cur_name, 0.0, 0.0});
        return 0;
    }
    // Put the larger output dimension on M (C^T = B^T A^T swaps the operands).
    if (s.N > s.M && s.offC2.empty()) {
        std::swap(s.M, s.N);
        std::swap(s.a, s.b);
        std::swap(s.offA, s.offB);
        std::swap(s.conjA, s.conjB);
        std::vector<int> ra = s.colB, ca = s.rowB, rb = s.colA, cb = s.rowA;
        s.rowA = ra; s.colA = ca; s.rowB = rb; s.colB = cb;
        std::swap(s.rowC, s.colC);
    }
    // Every element a launch can touch must lie inside its buffer.
    auto span = [](const std::vector<long long>& off, const std::vector<int>& r, const std::vector<int>& c) {
        long long lo = 0, hi = 0;
        if (off.empty() || r.empty() || c.empty()) return std::make_pair(-1LL, -1LL);
        lo = *std::min_element(off.begin(), off.end()) + *std::min_element(r.begin(), r.end()) + *std::min_element(c.begin(), c.end());
        hi = *std::max_element(off.begin(), off.end()) + *std::max_element(r.begin(), r.end()) + *std::max_element(c.begin(), c.end());
        return std::make_pair(lo, hi);
    };
    if ((long long)s.offA.size() != (long long)s.nbatch * s.nchunk || (long long)s.offB.size() != (long long)s.nbatch * s.nchunk ||
        (long long)s.offC.size() != s.nbatch || (int)s.rowA.size() != s.M || (int)s.colA.size() != s.K ||
        (int)s.rowB.size() != s.K || (int)s.colB.size() != s.N || (int)s.rowC.size() != s.M || (int)s.colC.size() != s.N)
        return CCSD_ERR_INVALID;
    const std::pair<long long, long long> sa = span(s.offA, s.rowA, s.colA), sb = span(s.offB, s.rowB, s.colB),
                                          sc = span(s.offC, s.rowC, s.colC);
    if (sa.first < 0 || sa.second >= h->bufsize[s.a] || sb.first < 0 || sb.second >= h->bufsize[s.b] ||
        sc.first < 0 || sc.second >= h->bufsize[s.c]) {
        snprintf(g_errbuf, sizeof g_errbuf, "plan %zu out of bounds", h->gemms.size());
        return CCSD_ERR_INVALID;
    }
    if (!s.nchunk_b.empty()) {
        if ((long long)s.nchunk_b.size() != s.nbatch) return CCSD_ERR_INVALID;
        for (int x : s.nchunk_b) if (x < 0 || x > s.nchunk) return CCSD_ERR_INVALID;
    }
    if (!s.offC2.empty()) {
        if ((long long)s.offC2.size() != s.nbatch || (int)s.colC2.size() != s.N) return CCSD_ERR_INVALID;
        const std::pair<long long, long long> s2 = span(s.offC2, s.rowC, s.colC2);
        if (s2.first < 0 || s2.second >= h->bufsize[s.c]) return CCSD_ERR_INVALID;
    }
    GemmPlan p{};
    p.a = s.a; p.b = s.b; p.c = s.c;
    // affine tables: the index arithmetic replaces the table loads in the kernel
    auto affine = [](const std::vector<int>& t, int& stride) {
        if (t.size() < 2) { stride = 0; return true; }
        const long long d = (long long)t[1] - t[0];
        if (d < INT_MIN || d > INT_MAX) return false;
        for (size_t i = 2; i < t.size(); ++i) if ((long long)t[i] - t[i - 1] != d) return false;
        stride = (int)d;
        return true;
    };
    {
        GemmArgs& g0 = p.args;
        g0.affA = affine(s.rowA, g0.rAs) && affine(s.colA, g0.cAs) ? 1 : 0;
        g0.affB = affine(s.rowB, g0.rBs) && affine(s.colB, g0.cBs) ? 1 : 0;
        g0.a0 = g0.affA ? (long long)s.rowA[0] + s.colA[0] : 0;
        g0.b0 = g0.affB ? (long long)s.rowB[0] + s.colB[0] : 0;
    }
    if (s.N >= 48) p.cfg = CFG_64x64;
    else if (s.N > 16) p.cfg = CFG_64x32;
    else if (s.M > 64) p.cfg = CFG_128x16;
    else if (s.M > 16) p.cfg = s.K >= 32 ? CFG_32x16K : CFG_32x16;
    else p.cfg = s.K >= 32 ? CFG_16x16K : CFG_16x16;
    GemmArgs& g = p.args;
    g.M = s.M; g.N = s.N; g.K = s.K; g.nbatch = s.nbatch; g.nchunk = s.nchunk;
    g.conjA = s.conjA; g.conjB = s.conjB; g.accumulate = s.acc ? 1 : 0;
    g.alpha_re = s.ar; g.alpha_im = s.ai;
    g.tiles_m = (s.M + CFG_BM[p.cfg] - 1) / CFG_BM[p.cfg];
    g.tiles_n = (s.N + CFG_BN[p.cfg] - 1) / CFG_BN[p.cfg];
    const long long ctas = (long long)g.tiles_m * g.tiles_n * s.nbatch;
    int nsplit = 1;
    if (ctas < 2 * kSMs && s.nchunk > 1) {
        nsplit = (int)std::min<long long>(s.nchunk, (4 * kSMs + ctas - 1) / ctas);
    }
    g.chunks_per_split = (s.nchunk + nsplit - 1) / nsplit;
    g.nsplit = (s.nchunk + g.chunks_per_split - 1) / g.chunks_per_split;
    if (g.nsplit > 1) work_need = std::max(work_need, (size_t)g.nsplit * s.nbatch * s.M * s.N);
    p.blocks = (int)ctas;
    g.offA = upload(al, s.offA, h->st); g.offB = upload(al, s.offB, h->st); g.offC = upload(al, s.offC, h->st);
    g.rowA = upload(al, s.rowA, h->st); g.colA = upload(al, s.colA, h->st);
    g.rowB = upload(al, s.rowB, h->st); g.colB = upload(al, s.colB, h->st);
    g.rowC = upload(al, s.rowC, h->st); g.colC = upload(al, s.colC, h->st);
    g.nchunk_b = s.nchunk_b.empty() ? nullptr : upload(al, s.nchunk_b, h->st);
    g.offC2 = s.offC2.empty() ? nullptr : upload(al, s.offC2, h->st);
    g.colC2 = s.colC2.empty() ? nullptr : upload(al, s.colC2, h->st);
    if (al.err) return al.err;
    // FP32 instance (mixed form): an FP32 partial sum runs over at most kFp32Chain terms
    // (or one momentum chunk); the chunk partials are added in FP64 by the split-K
    // reduction, so the FP32 rounding error stays that of a short sum
    p.args32 = g;
    {
        const long long kFp32Chain = 8192;
        GemmArgs& g32 = p.args32;
        if ((long long)g32.chunks_per_split * s.K > kFp32Chain && s.nchunk > 1) {
            g32.chunks_per_split = (int)std::max<long long>(1, kFp32Chain / std::max(1, s.K));
            g32.nsplit = (s.nchunk + g32.chunks_per_split - 1) / g32.chunks_per_split;
        }   // its split-K workspace is sized in setup_handle, for the steps that run in FP32
    }
    h->gemms.push_back(p);
    double chunks = (double)s.nchunk * s.nbatch;
    if (!s.nchunk_b.empty()) { chunks = 0.0; for (int x : s.nchunk_b) chunks += x; }
    h->seq.push_back({0, (int)h->gemms.size() - 1, h->cur_name, 8.0 * s.M * (double)s.N * s.K * chunks, 0.0});
    return 0;
}

int add_copy(ccsd_ctx* h, int dst, int src, long long n, int conj) {
    if (n > h->bufsize[dst] || n > h->bufsize[src]) return CCSD_ERR_INVALID;
    h->copies.push_back({dst, src, n, conj});
    h->seq.push_back({1, (int)h->copies.size() - 1, h->cur_name, 0.0, 32.0 * (double)n});
    return 0;
}

int add_perm(ccsd_ctx* h, Alloc& al, int dst, int src, int n0, int n1, int n2, int n3,
             int d0, int d1, int d2, int d3, int s0, int s1, int s2, int s3,
             const std::vector<long long>& offD, const std::vector<long long>& offS) {
    {
        const long long dmax = (long long)(n0 - 1) * d0 + (long long)(n1 - 1) * d1 + (long long)(n2 - 1) * d2 + (long long)(n3 - 1) * d3;
        const long long smax = (long long)(n0 - 1) * s0 + (long long)(n1 - 1) * s1 + (long long)(n2 - 1) * s2 + (long long)(n3 - 1) * s3;
        for (size_t i = 0; i < offD.size(); ++i)
            if (offD[i] < 0 || offS[i] < 0 || offD[i] + dmax >= h->bufsize[dst] || offS[i] + smax >= h->bufsize[src]) return CCSD_ERR_INVALID;
    }
    PermPlan pp{};
    pp.dst = dst; pp.src = src;
    pp.p.n0 = n0; pp.p.n1 = n1; pp.p.n2 = n2; pp.p.n3 = n3;
    pp.p.d0 = d0; pp.p.d1 = d1; pp.p.d2 = d2; pp.p.d3 = d3;
    pp.p.s0 = s0; pp.p.s1 = s1; pp.p.s2 = s2; pp.p.s3 = s3;
    pp.p.nbatch = (int)offD.size();
    pp.p.offD = upload(al, offD, h->st);
    pp.p.offS = upload(al, offS, h->st);
    if (al.err) return al.err;
    h->perms.push_back(pp);
    h->seq.push_back({2, (int)h->perms.size() - 1, h->cur_name, 0.0, 32.0 * (double)offD.size() * n0 * n1 * n2 * n3});
    return 0;
}

// Driver entry point for TMA descriptors (no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {     // resolved once, thread-safe
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)f;
        cudaGetLastError();
        return (PFN_cuTensorMapEncodeTiled_v12000)nullptr;
    }();
    return fn;
}

// 2D fp32 tensor [rows][kpad] with a (TC_BK x box_rows) box and 64-byte swizzle.
int encode_map(CUtensorMap* m, const float* base, long long rows, int kpad, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return CCSD_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 4};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : CCSD_ERR_CUDA;
}

// The Ozaki operand: `planes` BF16 slice planes of rows x kpad, stacked as one 2D view.
int encode_map_bf16(CUtensorMap* m, const uint16_t* base, long long rows, int kpad, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return CCSD_ERR_CUDA;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : CCSD_ERR_CUDA;
}

// Step mode of a tensor-core step of the operand set being added.
int tc_mode(const ccsd_ctx* h) { return h->cur_oz ? 5 : 2; }

// A tensor-core operand: split-TF32 parts (big, small: rows x kpad floats each), or for
// the Ozaki form BF16 slice planes (sl: planes x rows x kpad) and row scales (sc).
struct TcBuf { float* big; float* small; long long rows; int kpad; uint16_t* sl = nullptr; float* sc = nullptr; };

int tc_alloc(ccsd_ctx* h, Alloc& al, TcBuf& t, long long rows, int kpad) {
    t.rows = rows; t.kpad = kpad;
    if (h->cur_oz) {
        const size_t bytes = (size_t)rows * kpad * 2 * h->oz_slices;
        t.big = t.small = nullptr;
        t.sl = (uint16_t*)al.get(bytes);
        t.sc = (float*)al.get((size_t)rows * 4);
        if (al.err) return al.err;
        if (!al.dry && cudaMemsetAsync(t.sl, 0, bytes, h->st) != cudaSuccess) return CCSD_ERR_CUDA;
        return 0;
    }
    t.big = (float*)al.get((size_t)rows * kpad * 4);
    t.small = (float*)al.get((size_t)rows * kpad * 4);
    if (al.err) return al.err;
    if (!al.dry) {
        // padding columns must read as zero; the embed kernels write only the others
        if (cudaMemsetAsync(t.big, 0, (size_t)rows * kpad * 4, h->st) != cudaSuccess ||
            cudaMemsetAsync(t.small, 0, (size_t)rows * kpad * 4, h->st) != cudaSuccess) return CCSD_ERR_CUDA;
    }
    return 0;
}

int add_embed(ccsd_ctx* h, Alloc& al, int src, const TcBuf& dst, int mode, int R, int Kc,
              const std::vector<long long>& srcoff, const std::vector<int>& srow, const std::vector<int>& scol,
              bool constant, bool conj = false) {
    if (conj && !h->cur_oz) return CCSD_ERR_INVALID;
    const long long nblk = (long long)srcoff.size();
    if ((int)srow.size() != R || (int)scol.size() != Kc || 2 * Kc > dst.kpad) return CCSD_ERR_INVALID;
    const long long hi = *std::max_element(srcoff.begin(), srcoff.end()) + *std::max_element(srow.begin(), srow.end()) +
                         *std::max_element(scol.begin(), scol.end());
    const long long lo = *std::min_element(srcoff.begin(), srcoff.end()) + *std::min_element(srow.begin(), srow.end()) +
                         *std::min_element(scol.begin(), scol.end());
    if (lo < 0 || hi >= h->bufsize[src]) { refuse("an operand gather offset is out of range (32-bit tables)"); return CCSD_ERR_INVALID; }
    if (nblk * R * (mode == 0 ? 1 : 2) > dst.rows) { refuse("an embedded operand exceeds its buffer"); return CCSD_ERR_INVALID; }
    EmbedPlan e{};
    e.src = src;
    e.a.srcoff = upload(al, srcoff, h->st);
    e.a.srow = upload(al, srow, h->st);
    e.a.scol = upload(al, scol, h->st);
    if (al.err) return al.err;
    e.a.big = dst.big; e.a.small = dst.small;
    e.a.nblk = (int)nblk; e.a.R = R; e.a.Kc = Kc; e.a.Kpad = dst.kpad; e.a.mode = mode;
    if (h->cur_oz) {
        e.oz = true;
        e.z.srcoff = e.a.srcoff; e.z.srow = e.a.srow; e.z.scol = e.a.scol;
        e.z.sl = dst.sl; e.z.sc = dst.sc; e.z.rows = dst.rows;
        e.z.nblk = (int)nblk; e.z.R = R; e.z.Kc = Kc; e.z.Kpad = dst.kpad; e.z.mode = mode;
        e.z.slices = h->oz_slices;
        e.z.conj = conj ? 1 : 0;
    }
    h->embeds.push_back(e);
    if (constant) {
        h->const_embeds.push_back((int)h->embeds.size() - 1);
    } else {
        Step st{5, (int)h->embeds.size() - 1, h->cur_name, 0.0, (16.0 + (mode == 0 ? 16.0 : 32.0)) * nblk * R * Kc};
        st.mode = tc_mode(h);
        h->seq.push_back(st);
    }
    return 0;
}

int add_tc(ccsd_ctx* h, Alloc& al, const TcBuf& A, const TcBuf& B, int c, int M, int Nr, int nbatch, int nchunk,
           const std::vector<int>& rowA, const std::vector<int>& rowB, const std::vector<long long>& offC,
           const std::vector<int>& colC, double alpha, int nterms,
           const std::vector<int>& nchunk_b = {}, const std::vector<long long>& offC2 = {},
           const std::vector<int>& colC2 = {}, double alpha_im = 0.0, bool overwrite = false,
           const std::vector<int>& rowC = {}) {
    // output row m of batch b starts at offC[b * M + m], or (rowC given) at offC[b] + rowC[m]
    const bool oz = h->cur_oz;
    if (A.kpad != B.kpad || A.kpad % (oz ? OZ_BK : TC_BK)) return CCSD_ERR_INVALID;
    if (!oz && (alpha_im != 0.0 || overwrite || !rowC.empty())) return CCSD_ERR_INVALID;
    if (oz && ((long long)h->oz_slices * A.rows > INT_MAX || (long long)h->oz_slices * B.rows > INT_MAX)) {
        refuse("a tensor-core operand exceeds 2^31 rows (32-bit row indices)");
        return CCSD_ERR_INVALID;
    }
    const long long noff = rowC.empty() ? (long long)nbatch * M : nbatch;
    if ((long long)rowA.size() != (long long)nbatch * nchunk || (long long)rowB.size() != (long long)nbatch * nchunk ||
        (long long)offC.size() != noff || (int)colC.size() * 2 != Nr || (!rowC.empty() && (int)rowC.size() != M))
        return CCSD_ERR_INVALID;
    for (int x : rowA) if (x < 0 || x >= A.rows) { refuse("a tensor-core operand row index is out of range (32-bit row indices)"); return CCSD_ERR_INVALID; }
    for (int x : rowB) if (x < 0 || x >= B.rows) { refuse("a tensor-core operand row index is out of range (32-bit row indices)"); return CCSD_ERR_INVALID; }
    const long long rhi = rowC.empty() ? 0 : *std::max_element(rowC.begin(), rowC.end());
    const long long rlo = rowC.empty() ? 0 : *std::min_element(rowC.begin(), rowC.end());
    const long long chi = *std::max_element(offC.begin(), offC.end()) + rhi + *std::max_element(colC.begin(), colC.end());
    const long long clo = *std::min_element(offC.begin(), offC.end()) + rlo + *std::min_element(colC.begin(), colC.end());
    if (clo < 0 || chi >= h->bufsize[c]) { refuse("a tensor-core output offset is out of range (32-bit tables)"); return CCSD_ERR_INVALID; }
    if (!nchunk_b.empty()) {
        if ((long long)nchunk_b.size() != nbatch) return CCSD_ERR_INVALID;
        for (int x : nchunk_b) if (x < 0 || x > nchunk) return CCSD_ERR_INVALID;
    }
    if (!offC2.empty()) {
        if (offC2.size() != offC.size() || colC2.size() != colC.size()) return CCSD_ERR_INVALID;
        const long long h2 = *std::max_element(offC2.begin(), offC2.end()) + rhi + *std::max_element(colC2.begin(), colC2.end());
        const long long l2 = *std::min_element(offC2.begin(), offC2.end()) + rlo + *std::min_element(colC2.begin(), colC2.end());
        if (l2 < 0 || h2 >= h->bufsize[c]) { refuse("a tensor-core output offset is out of range (32-bit tables)"); return CCSD_ERR_INVALID; }
    }
    TcPlan t{};
    t.c = c;
    TcArgs& a = t.a;
    a.rowA = upload(al, rowA, h->st); a.rowB = upload(al, rowB, h->st);
    a.offC = upload(al, offC, h->st); a.colC = upload(al, colC, h->st);
    a.nchunk_b = nchunk_b.empty() ? nullptr : upload(al, nchunk_b, h->st);
    a.offC2 = offC2.empty() ? nullptr : upload(al, offC2, h->st);
    a.colC2 = colC2.empty() ? nullptr : upload(al, colC2, h->st);
    if (al.err) return al.err;
    a.err = h->tc_err;
    a.spin_limit = TC_SPIN_LIMIT;
    a.skip_stage = -1;
    a.M = M; a.Nr = Nr; a.nchunk = nchunk; a.kstages = A.kpad / TC_BK; a.nterms = nterms;
    a.tiles_m = (M + TC_BM - 1) / TC_BM; a.tiles_n = (Nr + TC_BN - 1) / TC_BN;
    a.alpha_re = alpha; a.alpha_im = 0.0;
    t.blocks = a.tiles_m * a.tiles_n * nbatch;
    if (oz) {
        t.oz = true;
        OzArgs& z = t.z;
        z.rowA = a.rowA; z.rowB = a.rowB; z.offC = a.offC; z.colC = a.colC;
        z.nchunk_b = a.nchunk_b; z.offC2 = a.offC2; z.colC2 = a.colC2;
        z.err = a.err; z.spin_limit = a.spin_limit; z.skip_stage = -1;
        z.scA = A.sc; z.scB = B.sc; z.rowsA = (int)A.rows; z.rowsB = (int)B.rows;
        z.M = M; z.Nr = Nr; z.nchunk = nchunk; z.kstages = A.kpad / OZ_BK; z.slices = h->oz_slices;
        z.tiles_m = (M + OZ_BM - 1) / OZ_BM; z.tiles_n = (Nr + OZ_BN - 1) / OZ_BN;
        z.alpha_re = alpha; z.alpha_im = alpha_im; z.overwrite = overwrite ? 1 : 0;
        z.rowC = rowC.empty() ? nullptr : upload(al, rowC, h->st);
        if (al.err) return al.err;
        z.nbatch = nbatch;
        // too few tiles for the 152 SMs: split each tile's (chunk, window) units over CTAs
        const long long tiles = (long long)z.tiles_m * z.tiles_n * nbatch;
        const int units = nchunk * oz_nwin(z.kstages, h->oz_slices);
        z.nsplit = 1;
        if (tiles < 2 * kSMs) z.nsplit = (int)std::min<long long>(std::min(units, OZ_MAX_SPLIT), (2 * kSMs + tiles - 1) / tiles);
        t.blocks = (int)(tiles * z.nsplit);
        if (z.nsplit > 1)
            h->oz_work_elems = std::max(h->oz_work_elems, (long long)z.nsplit * nbatch * M * (Nr / 2));
        if (!al.dry) {
            int rc;
            if ((rc = encode_map_bf16(&t.mA_big, A.sl, A.rows * h->oz_slices, A.kpad, OZ_BM)) ||
                (rc = encode_map_bf16(&t.mB_big, B.sl, B.rows * h->oz_slices, B.kpad, OZ_BN)))
                return rc;
        }
    } else if (!al.dry) {
        int rc;
        if ((rc = encode_map(&t.mA_big, A.big, A.rows, A.kpad, TC_BM)) || (rc = encode_map(&t.mA_small, A.small, A.rows, A.kpad, TC_BM)) ||
            (rc = encode_map(&t.mB_big, B.big, B.rows, B.kpad, TC_BN)) || (rc = encode_map(&t.mB_small, B.small, B.rows, B.kpad, TC_BN)))
            return rc;
    }
    h->tcs.push_back(t);
    double chunks = (double)nchunk * nbatch;
    if (!nchunk_b.empty()) { chunks = 0.0; for (int x : nchunk_b) chunks += x; }
    Step st{6, (int)h->tcs.size() - 1, h->cur_name, 8.0 * (double)M * (Nr / 2) * (A.kpad / 2) * chunks, 0.0};
    st.mode = tc_mode(h);
    h->seq.push_back(st);
    return 0;
}

void add_zero(ccsd_ctx* h, int buf) {
    Step st{7, buf, h->cur_name, 0.0, 16.0 * (double)h->bufsize[buf]};
    st.mode = tc_mode(h);
    h->seq.push_back(st);
}

dim3 ew_grid(long long n);
dim3 row_grid(long long rows);

// Ozaki form: every remaining FP64 GEMM step with at least OZ_CONVERT_FLOPS of work that
// the cost model below finds faster on the tensor cores than in the double-float engine
// gets a tensor-core alternative (the GEMM step stays for native FP64 iterations, mode 1).  The
// batches are split into groups whose distinct operand blocks fit the shared operand
// buffers; each group is embedded just before its GEMM (stream order keeps the buffers
// intact while it runs).  In the pooled layout the buffers are the tensor-core pools; else
// two buffers of at most OZ_GENERIC_CAP elements per slice plane are allocated here.
constexpr double OZ_CONVERT_FLOPS = 5e8;
// cost model of the conversion (measured on GB300: the per-CTA fixed cost of a launch of
// oz_gemm_kernel, the time of one slice-pair product of a 128 x 64 tile over a K slice of
// 64, embedding bandwidth, and the rate of the double-float GEMM engine on the skinny
// shapes it is left with, 1.3 .. 2.4 TFLOP/s)
constexpr double OZ_CTA_SECONDS = 8e-6;
constexpr double OZ_PAIR_SECONDS = 0.11e-6;
constexpr double OZ_EMBED_BPS = 2e12;
constexpr double OZ_DF_FLOPS = 1.5e12;
constexpr long long OZ_GENERIC_CAP = 1LL << 28;

int oz_convert_gemms(ccsd_ctx* h, Alloc& al, std::map<int, GemmSpec>& specs, bool pooled, float* pool_a,
                     float* pool_b, long long pool_ae, long long pool_be, float* pool_asc, float* pool_bsc,
                     long long pool_ar, long long pool_br) {
    struct Cand { int gi; int kpad; long long needA, needB, rowsA, rowsB; };
    std::map<int, Cand> cand;                  // by plan index of the FP64 GEMM
    long long maxA = 0, maxB = 0, maxRA = 0, maxRB = 0;
    for (const Step& st : h->seq) {
        if (st.kind != 0 || st.mode != 0 || st.flops < OZ_CONVERT_FLOPS) continue;
        auto it = specs.find(st.idx);
        if (it == specs.end() || it->second.nbatch == 0) continue;
        GemmSpec& s = it->second;
        // orientation: C^T = B^T A^T when that needs fewer tiles (rows M, real columns 2N)
        auto tiles = [](long long m, long long n) { return ((m + OZ_BM - 1) / OZ_BM) * ((2 * n + OZ_BN - 1) / OZ_BN); };
        if (s.offC2.empty() && tiles(s.N, s.M) < tiles(s.M, s.N)) {
            std::swap(s.M, s.N);
            std::swap(s.a, s.b);
            std::swap(s.offA, s.offB);
            std::swap(s.conjA, s.conjB);
            std::vector<int> ra = s.colB, ca = s.rowB, rb = s.colA, cb = s.rowA;
            s.rowA = ra; s.colA = ca; s.rowB = rb; s.colB = cb;
            std::swap(s.rowC, s.colC);
        }
        const int kpad = (2 * s.K + OZ_BK - 1) / OZ_BK * OZ_BK;
        std::vector<long long> ua(s.offA), ub(s.offB);
        std::sort(ua.begin(), ua.end()); ua.erase(std::unique(ua.begin(), ua.end()), ua.end());
        std::sort(ub.begin(), ub.end()); ub.erase(std::unique(ub.begin(), ub.end()), ub.end());
        // worth it?  Tensor-core estimate: the launch's waves of CTAs (with the kernel's own
        // split of small launches), each CTA a fixed cost plus its slice-pair products over
        // its K slices (padding included), plus the operand embedding at HBM speed; the
        // alternative is the double-float GEMM engine (algorithmic flops at its rate).
        const long long ntile = tiles(s.M, s.N) * s.nbatch;
        const int kst = kpad / OZ_BK;
        const long long units = (long long)s.nchunk * oz_nwin(kst, h->oz_slices);
        const long long nsplit = ntile < 2 * kSMs ? std::min<long long>(std::min<long long>(units, OZ_MAX_SPLIT),
                                                                          (2 * kSMs + ntile - 1) / ntile) : 1;
        const double waves = (double)((ntile * nsplit + kSMs - 1) / kSMs);
        const double pairs = h->oz_slices * (h->oz_slices + 1) / 2;
        const double per_cta = OZ_CTA_SECONDS + (double)s.nchunk * kst / nsplit * pairs * OZ_PAIR_SECONDS;
        const double emb = ((double)ua.size() * s.M + (double)ub.size() * 2 * s.N) * kpad * 2.0 * h->oz_slices;
        const double t_tc = waves * per_cta + emb / OZ_EMBED_BPS;
        const double t_df = st.flops / OZ_DF_FLOPS;
        if (t_tc > 0.7 * t_df) continue;
        // the largest single batch must fit: its chunks' A blocks and B blocks
        const long long ra = (long long)s.nchunk * s.M, rb = (long long)s.nchunk * 2 * s.N;
        cand[st.idx] = Cand{st.idx, kpad, ra * kpad, rb * kpad, ra, rb};
        // whole-GEMM sizes (distinct blocks) bound what a generic buffer needs
        maxA = std::max(maxA, (long long)ua.size() * s.M * kpad);
        maxB = std::max(maxB, (long long)ub.size() * 2 * s.N * kpad);
        maxRA = std::max(maxRA, (long long)ua.size() * s.M);
        maxRB = std::max(maxRB, (long long)ub.size() * 2 * s.N);
    }
    if (cand.empty()) return 0;
    uint16_t *ga = nullptr, *gb = nullptr;
    float *gasc = nullptr, *gbsc = nullptr;
    long long capA, capB, capRA, capRB;
    if (pooled) {
        ga = (uint16_t*)pool_a; gb = (uint16_t*)pool_b; gasc = pool_asc; gbsc = pool_bsc;
        capA = pool_ae; capB = pool_be; capRA = pool_ar; capRB = pool_br;
    } else {
        capA = std::min(maxA, OZ_GENERIC_CAP); capB = std::min(maxB, OZ_GENERIC_CAP);
        for (auto& kv : cand) { capA = std::max(capA, kv.second.needA); capB = std::max(capB, kv.second.needB); }
        capRA = maxRA; capRB = maxRB;
        TcBuf ta{}, tb{};
        int rc;
        if ((rc = tc_alloc(h, al, ta, capA / OZ_BK + 1, OZ_BK)) || (rc = tc_alloc(h, al, tb, capB / OZ_BK + 1, OZ_BK)))
            return rc;
        ga = ta.sl; gb = tb.sl;
        gasc = (float*)al.get((size_t)capRA * 4);
        gbsc = (float*)al.get((size_t)capRB * 4);
        if (al.err) return al.err;
    }
    std::vector<Step> old;
    old.swap(h->seq);
    const char* saved_name = h->cur_name;
    for (const Step& st : old) {
        auto it = cand.find(st.kind == 0 ? st.idx : -1);
        if (st.kind != 0 || st.mode != 0 || it == cand.end() || it->second.needA > capA || it->second.needB > capB ||
            it->second.rowsA > capRA || it->second.rowsB > capRB) {
            h->seq.push_back(st);
            continue;
        }
        Step f = st;
        f.mode = 1;                             // the FP64 GEMM: native FP64 iterations only
        h->seq.push_back(f);
        h->cur_name = st.name;
        const GemmSpec& s = specs.at(st.idx);
        const int kpad = it->second.kpad;
        int b0 = 0;
        while (b0 < s.nbatch) {
            // a group of batches whose distinct blocks fit the buffers
            std::map<long long, int> ia, ib;       // block offset -> block index in the group
            int b1 = b0;
            while (b1 < s.nbatch) {
                // blocks this batch would add
                std::vector<long long> newa, newb;
                for (int c = 0; c < s.nchunk; ++c) {
                    const long long xa = s.offA[(size_t)b1 * s.nchunk + c], xb = s.offB[(size_t)b1 * s.nchunk + c];
                    if (!ia.count(xa) && std::find(newa.begin(), newa.end(), xa) == newa.end()) newa.push_back(xa);
                    if (!ib.count(xb) && std::find(newb.begin(), newb.end(), xb) == newb.end()) newb.push_back(xb);
                }
                const long long ra = (long long)(ia.size() + newa.size()) * s.M;
                const long long rb = (long long)(ib.size() + newb.size()) * 2 * s.N;
                if (b1 > b0 && (ra * kpad > capA || rb * kpad > capB || ra > capRA || rb > capRB)) break;
                for (long long x : newa) ia.emplace(x, (int)ia.size());
                for (long long x : newb) ib.emplace(x, (int)ib.size());
                ++b1;
            }
            std::vector<long long> offa((size_t)ia.size()), offb((size_t)ib.size());
            for (auto& kv : ia) offa[(size_t)kv.second] = kv.first;
            for (auto& kv : ib) offb[(size_t)kv.second] = kv.first;
            TcBuf A{nullptr, nullptr, (long long)ia.size() * s.M, kpad, ga, gasc};
            TcBuf B{nullptr, nullptr, (long long)ib.size() * 2 * s.N, kpad, gb, gbsc};
            int rc;
            if ((rc = add_embed(h, al, s.a, A, 0, s.M, s.K, offa, s.rowA, s.colA, false, s.conjA)) ||
                (rc = add_embed(h, al, s.b, B, 1, s.N, s.K, offb, s.colB, s.rowB, false, s.conjB)))
                return rc;
            std::vector<int> rowa, rowb, nchb;
            std::vector<long long> oc, oc2;
            for (int b = b0; b < b1; ++b) {
                for (int c = 0; c < s.nchunk; ++c) {
                    rowa.push_back(ia.at(s.offA[(size_t)b * s.nchunk + c]) * s.M);
                    rowb.push_back(ib.at(s.offB[(size_t)b * s.nchunk + c]) * 2 * s.N);
                }
                oc.push_back(s.offC[b]);
                if (!s.offC2.empty()) oc2.push_back(s.offC2[b]);
                if (!s.nchunk_b.empty()) nchb.push_back(s.nchunk_b[b]);
            }
            if ((rc = add_tc(h, al, A, B, s.c, s.M, 2 * s.N, b1 - b0, s.nchunk, rowa, rowb, oc, s.colC, s.ar, 1, nchb,
                             oc2, s.offC2.empty() ? std::vector<int>{} : s.colC2, s.ai, !s.acc, s.rowC)))
                return rc;
            b0 = b1;
        }
    }
    h->cur_name = saved_name;
    return 0;
}

// Build the full residual plan.
int build_plan(ccsd_ctx* h, Alloc& al, size_t& work_need) {
    const KGrid& kg = h->kg;
    const int N = h->N, o = h->o, v = h->v;
    const long long ov = (long long)o * v, oo = (long long)o * o, vv = (long long)v * v;
    const long long S2 = oo * vv;                     // t2 / oovv / ovvo block
    const long long Soooo = oo * oo, Sooov = oo * ov, Sovvv = ov * vv, Svvvv = vv * vv;
    auto kk3 = [&](int a, int b, int c) { return ((long long)a * N + b) * N + c; };
    auto blk = [&](long long S, int a, int b, int c) { return kk3(a, b, c) * S; };
    int rc;
    std::map<int, GemmSpec> oz_specs;   // Ozaki form: the spec of every FP64 GEMM (by plan index)
    auto G = [&](GemmSpec& s) {
        if (h->cfg.precision == CCSD_OZAKI) oz_specs[(int)h->gemms.size()] = s;
        return finalize_gemm(h, al, s, work_need);
    };
    const bool mixed = h->cfg.precision == CCSD_MIXED;
    const bool oz = h->cfg.precision == CCSD_OZAKI;
    const bool tcp = mixed || oz;  // the plan has tensor-core variants of the large contractions
    // Tensor-core operand sets: split TF32 (mixed iterations) and/or Ozaki slices (Ozaki
    // iterations: the Ozaki form, or the mixed form's polish).  Both sets view the same
    // pools in the pooled layout; the two never run in the same iteration.
    struct TcSet {
        bool oz;
        int KQ, kpl, kplp, kpr, kpo;
        long long epb;                       // bytes per operand element
        TcBuf la, lap, lb, ra, rb, b1, ha, hb, h2a, h2b;
        long long lb_floats;                 // ladder B capacity (elements per part / slice plane)
        long long lad_max, lad_cap, pa, pb;  // sizes in elements per part / plane
    };
    std::vector<TcSet> sets;
    if (mixed) sets.push_back(TcSet{false});
    if (h->has_oz) sets.push_back(TcSet{true});
    bool pooled = false;          // tensor-core operands share two buffers, rewritten every residual
    float* pool_b = nullptr;      // the B-side pool (big part; the small part follows it)
    float* pool_a = nullptr;      // the A-side pool
    long long pool_ae = 0, pool_be = 0, pool_ar = 0, pool_br = 0;   // Ozaki capacity: elements, scale rows
    float* pool_asc = nullptr;
    float* pool_bsc = nullptr;    // Ozaki pools: row scales
    long long pool_b_bytes = 0;
    const long long nlt_vv = (long long)v * (v - 1) / 2;
    if (tcp) {
        const long long N3l = (long long)N * N * N;
        h->tc_err = (int*)al.get(sizeof(int));
        if (al.err) return al.err;
        if (mixed) {
            // complex64 copies: the inputs once here (unless stored so), t1 at the start of every
            // residual, t2 and tau~ by the tau kernel
            for (int bi = B_FOO_IN; bi <= B_T1; ++bi) {
                if (bi == B_T2 || h->in32[bi]) continue;
                h->shadow[bi] = (float2*)al.get((size_t)h->bufsize[bi] * 8);
                if (al.err) return al.err;
                if (!al.dry && bi != B_T1)
                    to_c64_kernel<<<ew_grid(h->bufsize[bi]), 256, 0, h->st>>>(ToC64Op{h->shadow[bi], h->buf[bi], h->bufsize[bi]});
            }
            h->shadow[B_T2] = (float2*)al.get((size_t)h->n2 * 8);
            h->shadow[B_TAUT] = (float2*)al.get((size_t)h->n2 * 8);
            if (al.err) return al.err;
        }
        if (!al.dry && cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->st) != cudaSuccess) return CCSD_ERR_CUDA;
        if (h->has_oz && !h->in32[B_OVVV]) {
            // the Ozaki W' kernel's t1 terms run in double-float: convert the constant ovvv once
            h->ovvv_df = (df2*)al.get((size_t)h->bufsize[B_OVVV] * sizeof(df2));
            if (al.err) return al.err;
            if (!al.dry)
                to_df2_kernel<<<ew_grid(h->bufsize[B_OVVV]), 256, 0, h->st>>>(h->ovvv_df, h->buf[B_OVVV],
                                                                             h->bufsize[B_OVVV]);
        }
        long long total_bytes = 0;
        for (TcSet& T : sets) {
            T.KQ = T.oz ? OZ_BK : TC_BK;      // row padding: one pipeline stage of K
            auto rnd = [&](long long x) { return (int)((x + T.KQ - 1) / T.KQ * T.KQ); };
            T.kpl = rnd(2 * vv); T.kplp = rnd(2 * nlt_vv); T.kpr = rnd(2 * ov); T.kpo = rnd(2 * oo);
            // bytes per operand element: split-TF32 big + small parts, or the Ozaki slice planes
            T.epb = T.oz ? 2LL * h->oz_slices : 8LL;
            // ladder B rows of the largest packed class
            long long lad_max = 0, lad_batch = 0;    // largest class, largest single (ka, kb) batch
            for (int diag_ab = 0; diag_ab < 2; ++diag_ab) for (int diag_ef = 0; diag_ef < 2; ++diag_ef) {
                const long long per_block = 2 * (diag_ab ? nlt_vv : vv) * (diag_ef ? T.kplp : T.kpl);
                long long blocks = 0;
                for (int ka = 0; ka < N; ++ka) for (int kb = ka; kb < N; ++kb) {
                    if ((ka == kb) != (diag_ab == 1)) continue;
                    const int S = kg.k4(ka, kb, 0);
                    long long nb = 0;
                    for (int ke = 0; ke < N; ++ke) { const int kf = kg.k4(S, 0, ke); if (diag_ef ? ke == kf : ke < kf) ++nb; }
                    blocks += nb;
                    lad_batch = std::max(lad_batch, nb * per_block);
                }
                lad_max = std::max(lad_max, blocks * per_block);
            }
            T.lad_max = lad_max;
            // 8 GB of operand (a third of the largest class in the lean layout), and never less
            // than one batch
            T.lad_cap = std::max(lad_batch, h->cfg.lean ? lad_max / 3 : (8LL << 30) / T.epb);
            // operand sizes (elements per part): A side (mode 0) and B side (mode 1)
            const long long fa[5] = {N3l * oo * T.kpl, N3l * oo * T.kplp, N3l * ov * T.kpr, N3l * oo * T.kpl,
                                     N3l * oo * T.kpo};
            const long long fb[4] = {N3l * 2 * ov * T.kpr, N3l * 2 * ov * T.kpr, N3l * 2 * oo * T.kpl,
                                     N3l * 2 * vv * T.kpo};
            long long total = std::min(lad_max, T.lad_cap);
            T.pa = 0; T.pb = std::min(lad_max, T.lad_cap);
            for (long long x : fa) { total += x; T.pa = std::max(T.pa, x); }
            for (long long x : fb) { total += x; T.pb = std::max(T.pb, x); }
            total_bytes += total * T.epb;
        }
        pooled = h->cfg.lean || total_bytes > (24LL << 30) * (long long)sets.size();
        if (!pooled) {
            for (TcSet& T : sets) {
                h->cur_oz = T.oz;
                T.lb_floats = std::max(1LL, std::min(T.lad_max, T.lad_cap));
                if ((rc = tc_alloc(h, al, T.la, N3l * oo, T.kpl)) ||
                    (rc = tc_alloc(h, al, T.lap, N3l * oo, std::max(T.kplp, T.KQ))) ||
                    (rc = tc_alloc(h, al, T.lb, T.lb_floats / T.kpl + 1, T.kpl)) ||
                    (rc = tc_alloc(h, al, T.ra, N3l * ov, T.kpr)) || (rc = tc_alloc(h, al, T.rb, N3l * 2 * ov, T.kpr)) ||
                    (rc = tc_alloc(h, al, T.b1, N3l * 2 * ov, T.kpr)) ||
                    (rc = tc_alloc(h, al, T.ha, N3l * oo, T.kpl)) || (rc = tc_alloc(h, al, T.hb, N3l * 2 * oo, T.kpl)) ||
                    (rc = tc_alloc(h, al, T.h2a, N3l * oo, T.kpo)) || (rc = tc_alloc(h, al, T.h2b, N3l * 2 * vv, T.kpo)))
                    return rc;
                T.lb_floats = T.lb.rows * T.kpl;
            }
        } else {
            // Large problems: every tensor-core step embeds its operands into one of two pools
            // just before its GEMM (stream order keeps them intact while it runs).  The B
            // pool also serves the FP64 ladder's W' slab, which only FP64 iterations use.
            long long bytes_a = 0, bytes_b = h->bufsize[B_WAB] * 16;
            for (TcSet& T : sets) {
                // the small part starts right after the big part: keep it 256-byte aligned (TMA
                // needs 16-byte aligned bases)
                T.pa = (T.pa + 63) / 64 * 64;
                T.pb = (T.pb + 63) / 64 * 64;
                bytes_a = std::max(bytes_a, T.pa * T.epb);
                bytes_b = std::max(bytes_b, T.pb * T.epb);
            }
            pool_a = (float*)al.get((size_t)bytes_a);
            pool_b = (float*)al.get((size_t)bytes_b);
            pool_b_bytes = bytes_b;
            if (al.err) return al.err;
            for (TcSet& T : sets) {
                // elements per part / plane the pools hold for this set
                const long long pa = bytes_a / T.epb / 64 * 64, pb = bytes_b / T.epb / 64 * 64;
                float* scA = nullptr;
                float* scB = nullptr;
                if (T.oz) {   // row scales of the largest A-side and B-side operands
                    const long long ra = N3l * std::max(oo, ov);
                    const long long rb = std::max({N3l * 2 * ov, N3l * 2 * oo, N3l * 2 * vv, pb / T.kpl + 1});
                    scA = (float*)al.get((size_t)ra * 4);
                    scB = (float*)al.get((size_t)rb * 4);
                    if (al.err) return al.err;
                    pool_ar = ra; pool_br = rb; pool_ae = pa; pool_be = pb; pool_asc = scA; pool_bsc = scB;
                }
                T.lb_floats = pb;
                const bool zo = T.oz;
                auto view = [zo](float* base, float* sc, long long floats, long long rows, int kpad) {
                    if (zo) {
                        TcBuf t{nullptr, nullptr, rows, kpad, (uint16_t*)base, sc};
                        return t;
                    }
                    TcBuf t{base, base + floats, rows, kpad};
                    return t;
                };
                T.la = view(pool_a, scA, pa, N3l * oo, T.kpl); T.lap = view(pool_a, scA, pa, N3l * oo, std::max(T.kplp, T.KQ));
                T.ra = view(pool_a, scA, pa, N3l * ov, T.kpr); T.ha = view(pool_a, scA, pa, N3l * oo, T.kpl);
                T.h2a = view(pool_a, scA, pa, N3l * oo, T.kpo);
                T.rb = view(pool_b, scB, pb, N3l * 2 * ov, T.kpr); T.b1 = view(pool_b, scB, pb, N3l * 2 * ov, T.kpr);
                T.hb = view(pool_b, scB, pb, N3l * 2 * oo, T.kpl); T.h2b = view(pool_b, scB, pb, N3l * 2 * vv, T.kpo);
                T.lb = view(pool_b, scB, pb, pb / T.kpl, T.kpl);
            }
            h->buf[B_WAB] = (double2*)pool_b;
        }
    }
    if (!pooled) {
        h->buf[B_WAB] = (double2*)al.get((size_t)h->bufsize[B_WAB] * 16);
        if (al.err) return al.err;
    }

    // ---------------- tau, tau~
    if (mixed) {
        Step st{9, B_T1, "tau", 0.0, 24.0 * h->n1};
        st.mode = 3;
        h->seq.push_back(st);
    }
    h->seq.push_back({3, 0, "tau", 0.0, 16.0 * (3.0 * h->n2 + h->n1)});

    h->cur_name = "F_ov";
    // ---------------- F~_ov (Eq. ori_F_ov): f_ov + sum t_r^c <p k r k^||g k c k^>
    if ((rc = add_copy(h, B_FOV, B_FOV_IN, (long long)N * ov, 0))) return rc;
    {
        GemmSpec s; s.a = B_OOVV; s.b = B_T1; s.c = B_FOV;
        s.M = (int)ov; s.N = 1; s.K = (int)ov; s.nbatch = N; s.nchunk = N;
        for (int k = 0; k < N; ++k) {
            for (int kh = 0; kh < N; ++kh) { s.offA.push_back(blk(S2, k, kh, k)); s.offB.push_back(kh * ov); }
            s.offC.push_back(k * ov);
        }
        s.rowA = tab({{o, ov * v}, {v, v}}); s.colA = tab({{o, vv}, {v, 1}});
        s.rowB = tab({{(int)ov, 1}}); s.colB = {0};
        s.rowC = tab({{(int)ov, 1}}); s.colC = {0};
        if ((rc = G(s))) return rc;
    }
    h->cur_name = "F_oo";
    // ---------------- F~_oo (Eq. ori_F_oo)
    if ((rc = add_copy(h, B_FOO, B_FOO_IN, (long long)N * oo, 0))) return rc;
    {   // + 1/2 sum_c f_p^c t_q^c
        GemmSpec s; s.a = B_FOV_IN; s.b = B_T1; s.c = B_FOO;
        s.M = o; s.N = o; s.K = v; s.nbatch = N; s.nchunk = 1; s.ar = 0.5;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * ov); s.offB.push_back(k * ov); s.offC.push_back(k * oo); }
        s.rowA = tab({{o, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{o, o}}); s.colC = tab({{o, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // + sum t_r^c(k^) <p k r k^||q k c k^>
        GemmSpec s; s.a = B_OOOV; s.b = B_T1; s.c = B_FOO;
        s.M = (int)oo; s.N = 1; s.K = (int)ov; s.nbatch = N; s.nchunk = N;
        for (int k = 0; k < N; ++k) {
            for (int kh = 0; kh < N; ++kh) { s.offA.push_back(blk(Sooov, k, kh, k)); s.offB.push_back(kh * ov); }
            s.offC.push_back(k * oo);
        }
        s.rowA = tab({{o, oo * v}, {o, v}}); s.colA = tab({{o, ov}, {v, 1}});
        s.rowB = tab({{(int)ov, 1}}); s.colB = {0};
        s.rowC = tab({{(int)oo, 1}}); s.colC = {0};
        if ((rc = G(s))) return rc;
    }
    {   // + 1/2 sum tau~_{q n}^{e f} <p n||e f>
        GemmSpec s; s.a = B_OOVV; s.b = B_TAUT; s.c = B_FOO;
        s.M = o; s.N = o; s.K = (int)(o * vv); s.nbatch = N; s.nchunk = N * N; s.ar = 0.5;
        for (int k = 0; k < N; ++k) {
            for (int kn = 0; kn < N; ++kn)
                for (int ke = 0; ke < N; ++ke) { s.offA.push_back(blk(S2, k, kn, ke)); s.offB.push_back(blk(S2, k, kn, ke)); }
            s.offC.push_back(k * oo);
        }
        s.rowA = tab({{o, o * vv}}); s.colA = tab({{(int)(o * vv), 1}});
        s.rowB = tab({{(int)(o * vv), 1}}); s.colB = tab({{o, o * vv}});
        s.rowC = tab({{o, o}}); s.colC = tab({{o, 1}});
        if ((rc = G(s))) return rc;
    }
    h->cur_name = "F_vv";
    // ---------------- F~_vv (Eq. ori_F_vv)
    if ((rc = add_copy(h, B_FVV, B_FVV_IN, (long long)N * vv, 0))) return rc;
    {   // - 1/2 sum_r f_r^h t_r^g
        GemmSpec s; s.a = B_T1; s.b = B_FOV_IN; s.c = B_FVV;
        s.M = v; s.N = v; s.K = o; s.nbatch = N; s.nchunk = 1; s.ar = -0.5;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * ov); s.offB.push_back(k * ov); s.offC.push_back(k * vv); }
        s.rowA = tab({{v, 1}}); s.colA = tab({{o, v}});
        s.rowB = tab({{o, v}}); s.colB = tab({{v, 1}});
        s.rowC = tab({{v, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // + sum t_r^c(k^) <g k r k^||h k c k^> = ovvv[k^,k,k^](r,g,c,h)
        GemmSpec s; s.a = B_OVVV; s.b = B_T1; s.c = B_FVV;
        s.M = (int)vv; s.N = 1; s.K = (int)ov; s.nbatch = N; s.nchunk = N;
        for (int k = 0; k < N; ++k) {
            for (int kh = 0; kh < N; ++kh) { s.offA.push_back(blk(Sovvv, kh, k, kh)); s.offB.push_back(kh * ov); }
            s.offC.push_back(k * vv);
        }
        s.rowA = tab({{v, vv}, {v, 1}}); s.colA = tab({{o, vv * v}, {v, v}});
        s.rowB = tab({{(int)ov, 1}}); s.colB = {0};
        s.rowC = tab({{(int)vv, 1}}); s.colC = {0};
        if ((rc = G(s))) return rc;
    }
    {   // - 1/2 sum tau~_{mn}^{g f} <m n||h f>
        GemmSpec s; s.a = B_TAUT; s.b = B_OOVV; s.c = B_FVV;
        s.M = v; s.N = v; s.K = (int)(oo * v); s.nbatch = N; s.nchunk = N * N; s.ar = -0.5;
        for (int k = 0; k < N; ++k) {
            for (int km = 0; km < N; ++km)
                for (int kn = 0; kn < N; ++kn) { s.offA.push_back(blk(S2, km, kn, k)); s.offB.push_back(blk(S2, km, kn, k)); }
            s.offC.push_back(k * vv);
        }
        s.rowA = tab({{v, v}}); s.colA = tab({{(int)oo, vv}, {v, 1}});
        s.rowB = tab({{(int)oo, vv}, {v, 1}}); s.colB = tab({{v, v}});
        s.rowC = tab({{v, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    h->cur_name = "F_prime";
    // ---------------- F' combinations used by T2
    if ((rc = add_copy(h, B_FVVP, B_FVV, (long long)N * vv, 0))) return rc;
    {   // F~^bf - 1/2 sum_r t_r^b F~_r^f
        GemmSpec s; s.a = B_T1; s.b = B_FOV; s.c = B_FVVP;
        s.M = v; s.N = v; s.K = o; s.nbatch = N; s.nchunk = 1; s.ar = -0.5;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * ov); s.offB.push_back(k * ov); s.offC.push_back(k * vv); }
        s.rowA = tab({{v, 1}}); s.colA = tab({{o, v}});
        s.rowB = tab({{o, v}}); s.colB = tab({{v, 1}});
        s.rowC = tab({{v, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    if ((rc = add_copy(h, B_FOOP, B_FOO, (long long)N * oo, 0))) return rc;
    {   // F~_nj + 1/2 sum_c t_j^c F~_n^c
        GemmSpec s; s.a = B_FOV; s.b = B_T1; s.c = B_FOOP;
        s.M = o; s.N = o; s.K = v; s.nbatch = N; s.nchunk = 1; s.ar = 0.5;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * ov); s.offB.push_back(k * ov); s.offC.push_back(k * oo); }
        s.rowA = tab({{o, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{o, o}}); s.colC = tab({{o, 1}});
        if ((rc = G(s))) return rc;
    }
    h->cur_name = "R1";
    // ---------------- R1 (Eq. ori_EqSingle); driver <a|f|i> = f_ov^*
    if ((rc = add_copy(h, B_R1, B_FOV_IN, (long long)N * ov, 1))) return rc;
    {   // + sum_c F~^{ac} t_i^c
        GemmSpec s; s.a = B_T1; s.b = B_FVV; s.c = B_R1;
        s.M = o; s.N = v; s.K = v; s.nbatch = N; s.nchunk = 1;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * ov); s.offB.push_back(k * vv); s.offC.push_back(k * ov); }
        s.rowA = tab({{o, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{v, v}});
        s.rowC = tab({{o, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // - sum_r t_r^a F~_{ri}
        GemmSpec s; s.a = B_FOO; s.b = B_T1; s.c = B_R1;
        s.M = o; s.N = v; s.K = o; s.nbatch = N; s.nchunk = 1; s.ar = -1.0;
        for (int k = 0; k < N; ++k) { s.offA.push_back(k * oo); s.offB.push_back(k * ov); s.offC.push_back(k * ov); }
        s.rowA = tab({{o, 1}}); s.colA = tab({{o, o}});
        s.rowB = tab({{o, v}}); s.colB = tab({{v, 1}});
        s.rowC = tab({{o, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // + sum F~_n^f(k^) t_{i k n k^}^{a k f k^}
        GemmSpec s; s.a = B_T2; s.b = B_FOV; s.c = B_R1;
        s.M = (int)ov; s.N = 1; s.K = (int)ov; s.nbatch = N; s.nchunk = N;
        for (int k = 0; k < N; ++k) {
            for (int kh = 0; kh < N; ++kh) { s.offA.push_back(blk(S2, k, kh, k)); s.offB.push_back(kh * ov); }
            s.offC.push_back(k * ov);
        }
        s.rowA = tab({{o, o * vv}, {v, v}}); s.colA = tab({{o, vv}, {v, 1}});
        s.rowB = tab({{(int)ov, 1}}); s.colB = {0};
        s.rowC = tab({{(int)ov, 1}}); s.colC = {0};
        if ((rc = G(s))) return rc;
    }
    {   // + sum t_r^c(k^) <a k r k^||i k c k^> = ovvo[k^,k,k^](r,a,c,i)
        GemmSpec s; s.a = B_OVVO; s.b = B_T1; s.c = B_R1;
        s.M = (int)ov; s.N = 1; s.K = (int)ov; s.nbatch = N; s.nchunk = N;
        for (int k = 0; k < N; ++k) {
            for (int kh = 0; kh < N; ++kh) { s.offA.push_back(blk(S2, kh, k, kh)); s.offB.push_back(kh * ov); }
            s.offC.push_back(k * ov);
        }
        s.rowA = tab({{o, 1}, {v, v * o}}); s.colA = tab({{o, vv * o}, {v, o}});
        s.rowB = tab({{(int)ov, 1}}); s.colB = {0};
        s.rowC = tab({{(int)ov, 1}}); s.colC = {0};
        if ((rc = G(s))) return rc;
    }
    {   // - 1/2 sum t_{mn}^{a f} <m n||i f>
        GemmSpec s; s.a = B_OOOV; s.b = B_T2; s.c = B_R1;
        s.M = o; s.N = v; s.K = (int)(oo * v); s.nbatch = N; s.nchunk = N * N; s.ar = -0.5;
        for (int k = 0; k < N; ++k) {
            for (int km = 0; km < N; ++km)
                for (int kn = 0; kn < N; ++kn) { s.offA.push_back(blk(Sooov, km, kn, k)); s.offB.push_back(blk(S2, km, kn, k)); }
            s.offC.push_back(k * ov);
        }
        s.rowA = tab({{o, v}}); s.colA = tab({{(int)oo, ov}, {v, 1}});
        s.rowB = tab({{(int)oo, vv}, {v, 1}}); s.colB = tab({{v, v}});
        s.rowC = tab({{o, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // + 1/2 sum t_{i n}^{e f} <a n||e f> = - 1/2 sum t_in^ef ovvv[kn,k,ke](n,a,e,f)
        GemmSpec s; s.a = B_T2; s.b = B_OVVV; s.c = B_R1;
        s.M = o; s.N = v; s.K = (int)(o * vv); s.nbatch = N; s.nchunk = N * N; s.ar = -0.5;
        for (int k = 0; k < N; ++k) {
            for (int kn = 0; kn < N; ++kn)
                for (int ke = 0; ke < N; ++ke) { s.offA.push_back(blk(S2, k, kn, ke)); s.offB.push_back(blk(Sovvv, kn, k, ke)); }
            s.offC.push_back(k * ov);
        }
        s.rowA = tab({{o, o * vv}}); s.colA = tab({{o, vv}, {(int)vv, 1}});
        s.rowB = tab({{o, vv * v}, {(int)vv, 1}}); s.colB = tab({{v, vv}});
        s.rowC = tab({{o, v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }

    h->cur_name = "R2_driver";
    // ---------------- R2 (Eq. ori_EqDouble); driver <ab||ij> = <ij||ab>^*
    if ((rc = add_copy(h, B_R2, B_OOVV, (long long)N * N * N * S2, 1))) return rc;
    const int N3 = N * N * N;
    h->cur_name = "hole_hole_W";
    // hole-hole: Whh = <mn||ij> + P(ij) t_j^c <mn||ic> + 1/2 tau_ij^ef <mn||ef>
    if ((rc = add_copy(h, B_WHH, B_OOOO, (long long)N3 * Soooo, 0))) return rc;
    {
        GemmSpec s; s.a = B_OOOV; s.b = B_T1; s.c = B_WHH;
        s.M = (int)(oo * o); s.N = o; s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int km = 0; km < N; ++km) for (int kn = 0; kn < N; ++kn) for (int ki = 0; ki < N; ++ki) {
            const int kj = kg.k4(km, kn, ki);
            s.offA.push_back(blk(Sooov, km, kn, ki)); s.offB.push_back(kj * ov); s.offC.push_back(blk(Soooo, km, kn, ki));
        }
        s.rowA = tab({{(int)(oo * o), v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{(int)(oo * o), o}}); s.colC = tab({{o, 1}});
        if ((rc = G(s))) return rc;
    }
    {
        GemmSpec s; s.a = B_OOOV; s.b = B_T1; s.c = B_WHH; s.ar = -1.0;
        s.M = (int)(oo * o); s.N = o; s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int km = 0; km < N; ++km) for (int kn = 0; kn < N; ++kn) for (int ki = 0; ki < N; ++ki) {
            const int kj = kg.k4(km, kn, ki);
            s.offA.push_back(blk(Sooov, km, kn, kj)); s.offB.push_back(ki * ov); s.offC.push_back(blk(Soooo, km, kn, ki));
        }
        s.rowA = tab({{(int)(oo * o), v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{(int)oo, oo}, {o, 1}}); s.colC = tab({{o, o}});
        if ((rc = G(s))) return rc;
    }
    // packed index pairs for the hole-hole contractions
    std::vector<int> vv_full = tab({{(int)vv, 1}}), vv_lt, oo_full = tab({{(int)oo, 1}}), oo_lt;
    for (int x = 0; x < v; ++x) for (int y = x + 1; y < v; ++y) vv_lt.push_back(x * v + y);
    for (int x = 0; x < o; ++x) for (int y = x + 1; y < o; ++y) oo_lt.push_back(x * o + y);
    auto swap_pair = [](int x, int n) { return (x % n) * n + x / n; };
    {   // Whh += 1/2 sum tau_ij^ef <mn||ef>, packed by antisymmetry in (e ke, f kf) and
        // (m km, n kn): ke < kf with all e f plus ke = kf with e < f (factor 2), and only
        // km < kn (all m n) or km = kn (m < n), mirrored as Whh(nm) = -Whh(mn).
        for (int diag_mn = 0; diag_mn < 2; ++diag_mn) for (int diag_ef = 0; diag_ef < 2; ++diag_ef) {
            GemmSpec s; s.a = B_TAU; s.b = B_OOVV; s.c = B_WHH; s.ar = 1.0;
            const std::vector<int>& kc = diag_ef ? vv_lt : vv_full;
            const std::vector<int>& nc = diag_mn ? oo_lt : oo_full;
            s.M = (int)oo; s.N = (int)nc.size(); s.K = (int)kc.size(); s.nchunk = N; s.nbatch = 0;
            for (int km = 0; km < N; ++km) for (int kn = km; kn < N; ++kn) {
                if ((km == kn) != (diag_mn == 1)) continue;
                const int S = kg.k4(km, kn, 0);
                std::vector<int> kes;
                for (int ke = 0; ke < N; ++ke) { const int kf = kg.k4(S, 0, ke); if (diag_ef ? ke == kf : ke < kf) kes.push_back(ke); }
                if (kes.empty() || nc.empty() || kc.empty()) continue;
                for (int ki = 0; ki < N; ++ki) {
                    const int kj = kg.k4(km, kn, ki);
                    for (int c = 0; c < N; ++c) {
                        const int ke = kes[std::min<size_t>(c, kes.size() - 1)];
                        s.offA.push_back(blk(S2, ki, kj, ke)); s.offB.push_back(blk(S2, km, kn, ke));
                    }
                    s.nchunk_b.push_back((int)kes.size());
                    s.offC.push_back(blk(Soooo, km, kn, ki));
                    s.offC2.push_back(blk(Soooo, kn, km, ki));
                    ++s.nbatch;
                }
            }
            s.rowA = tab({{(int)oo, vv}}); s.colA = kc;
            s.rowB = kc; for (int x : nc) s.colB.push_back(x * (int)vv);
            s.rowC = tab({{(int)oo, 1}});
            for (int x : nc) { s.colC.push_back(x * (int)oo); s.colC2.push_back(swap_pair(x, o) * (int)oo); }
            if ((rc = G(s))) return rc;
            if (tcp) h->seq.back().mode = 1;
        }
    }
    for (TcSet& T : sets) {
        h->cur_oz = T.oz;
        // X on tensor cores, one batch per momentum sum S = km + kn = ki + kj:
        // rows (km, mn) of <mn||ef> (constant operand), columns (ki, ij) of tau, K = (ke, ef)
        std::vector<long long> so;
        for (int S = 0; S < N; ++S) for (int ke = 0; ke < N; ++ke) for (int km = 0; km < N; ++km)
            so.push_back(blk(S2, km, kg.k4(S, 0, km), ke));
        if ((rc = add_embed(h, al, B_OOVV, T.ha, 0, (int)oo, (int)vv, so, tab({{(int)oo, vv}}), tab({{(int)vv, 1}}), !pooled)))
            return rc;
        so.clear();
        for (int S = 0; S < N; ++S) for (int ke = 0; ke < N; ++ke) for (int ki = 0; ki < N; ++ki)
            so.push_back(blk(S2, ki, kg.k4(S, 0, ki), ke));
        if ((rc = add_embed(h, al, B_TAU, T.hb, 1, (int)oo, (int)vv, so, tab({{(int)oo, vv}}), tab({{(int)vv, 1}}), false)))
            return rc;
        std::vector<int> ra, rb; std::vector<long long> oc;
        for (int S = 0; S < N; ++S) {
            for (int ke = 0; ke < N; ++ke) {
                ra.push_back((int)((((long long)S * N + ke) * N) * oo));
                rb.push_back((int)((((long long)S * N + ke) * N) * 2 * oo));
            }
            for (int km = 0; km < N; ++km)
                for (int mn = 0; mn < (int)oo; ++mn)
                    oc.push_back(((long long)km * N + kg.k4(S, 0, km)) * N * Soooo + mn * oo);
        }
        if ((rc = add_tc(h, al, T.ha, T.hb, B_WHH, (int)(N * oo), (int)(2 * N * oo), N, N, ra, rb, oc,
                         tab({{N, Soooo}, {(int)oo, 1}}), 0.5, 3))) return rc;
    }
    h->cur_name = "hole_hole";
    {   // R2 += 1/2 sum tau_mn^ab Whh_mnij, packed: (m km) < (n kn) over the sum
        // (factor 2) and (a ka) < (b kb) on the output with the mirror R2(ba) = -R2(ab).
        for (int diag_ab = 0; diag_ab < 2; ++diag_ab) for (int diag_mn = 0; diag_mn < 2; ++diag_mn) {
            GemmSpec s; s.a = B_WHH; s.b = B_TAU; s.c = B_R2; s.ar = 1.0;
            const std::vector<int>& kc = diag_mn ? oo_lt : oo_full;
            const std::vector<int>& nc = diag_ab ? vv_lt : vv_full;
            s.M = (int)oo; s.N = (int)nc.size(); s.K = (int)kc.size(); s.nchunk = N; s.nbatch = 0;
            for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) {
                const int S = kg.k4(ki, kj, 0);
                std::vector<int> kms;
                for (int km = 0; km < N; ++km) { const int kn = kg.k4(S, 0, km); if (diag_mn ? km == kn : km < kn) kms.push_back(km); }
                if (kms.empty() || nc.empty() || kc.empty()) continue;
                for (int ka = 0; ka < N; ++ka) {
                    const int kb = kg.k4(ki, kj, ka);
                    if (!(diag_ab ? ka == kb : ka < kb)) continue;
                    for (int c = 0; c < N; ++c) {
                        const int km = kms[std::min<size_t>(c, kms.size() - 1)];
                        const int kn = kg.k4(S, 0, km);
                        s.offA.push_back(blk(Soooo, km, kn, ki)); s.offB.push_back(blk(S2, km, kn, ka));
                    }
                    s.nchunk_b.push_back((int)kms.size());
                    s.offC.push_back(blk(S2, ki, kj, ka));
                    s.offC2.push_back(blk(S2, ki, kj, kb));
                    ++s.nbatch;
                }
            }
            s.rowA = tab({{(int)oo, 1}}); for (int x : kc) s.colA.push_back(x * (int)oo);
            for (int x : kc) s.rowB.push_back(x * (int)vv); s.colB = nc;
            s.rowC = tab({{(int)oo, vv}}); s.colC = nc;
            for (int x : nc) s.colC2.push_back(swap_pair(x, v));
            if ((rc = G(s))) return rc;
            if (tcp) h->seq.back().mode = 1;
        }
    }
    for (TcSet& T : sets) {
        h->cur_oz = T.oz;
        // R2 += 1/2 tau_mn^ab Whh_mnij on tensor cores, one batch per S = ki + kj:
        // rows (ki, ij) of Whh^T, columns (ka, ab) of tau, K = (km, mn)
        std::vector<long long> so;
        for (int S = 0; S < N; ++S) for (int km = 0; km < N; ++km) for (int ki = 0; ki < N; ++ki)
            so.push_back(blk(Soooo, km, kg.k4(S, 0, km), ki));
        if ((rc = add_embed(h, al, B_WHH, T.h2a, 0, (int)oo, (int)oo, so, tab({{(int)oo, 1}}), tab({{(int)oo, oo}}), false)))
            return rc;
        so.clear();
        for (int S = 0; S < N; ++S) for (int km = 0; km < N; ++km) for (int ka = 0; ka < N; ++ka)
            so.push_back(blk(S2, km, kg.k4(S, 0, km), ka));
        if ((rc = add_embed(h, al, B_TAU, T.h2b, 1, (int)vv, (int)oo, so, tab({{(int)vv, 1}}), tab({{(int)oo, vv}}), false)))
            return rc;
        std::vector<int> ra, rb; std::vector<long long> oc;
        for (int S = 0; S < N; ++S) {
            for (int km = 0; km < N; ++km) {
                ra.push_back((int)((((long long)S * N + km) * N) * oo));
                rb.push_back((int)((((long long)S * N + km) * N) * 2 * vv));
            }
            for (int ki = 0; ki < N; ++ki)
                for (int ij = 0; ij < (int)oo; ++ij)
                    oc.push_back(((long long)ki * N + kg.k4(S, 0, ki)) * N * S2 + ij * vv);
        }
        if ((rc = add_tc(h, al, T.h2a, T.h2b, B_R2, (int)(N * oo), (int)(2 * N * vv), N, N, ra, rb, oc,
                         tab({{N, S2}, {(int)vv, 1}}), 0.5, 3))) return rc;
    }
    // ladder: Wab = <ab||ef> - P(ab) t_r^b <a r||e f>, formed for slabs of momentum pairs
    // (ka <= kb; the packed ladder reads no others) into a bounded buffer, each slab
    // followed by its ladder contractions.  Slot p of a slab holds pair p's blocks
    // [p][ke](a,b,e,f).
    {
        std::vector<std::pair<int, int>> pairs;
        for (int ka = 0; ka < N; ++ka) for (int kb = ka; kb < N; ++kb) pairs.push_back({ka, kb});
        const long long pair_el = (long long)N * Svvvv;
        const int per_slab = (int)wab_pairs_per_slab(N, v, h->wab_cap_bytes);
        std::vector<int> pairs_full = tab({{(int)vv, 1}}), pairs_lt;
        for (int x = 0; x < v; ++x) for (int y = x + 1; y < v; ++y) pairs_lt.push_back(x * v + y);
        std::vector<int> swapped;                       // (a,b) -> (b,a) for every a, b
        for (int x = 0; x < v; ++x) for (int y = 0; y < v; ++y) swapped.push_back(y * v + x);
        for (size_t p0 = 0; p0 < pairs.size(); p0 += per_slab) {
            const size_t p1 = std::min(pairs.size(), p0 + per_slab);
            h->cur_name = "ladder_W";
            const size_t w_first = h->seq.size();
            {   // W'[p] = vvvv[ka][kb]: one contiguous run of N blocks per pair
                std::vector<long long> offD, offS;
                for (size_t p = p0; p < p1; ++p) {
                    offD.push_back((long long)(p - p0) * pair_el);
                    offS.push_back(((long long)pairs[p].first * N + pairs[p].second) * pair_el);
                }
                if ((rc = add_perm(h, al, B_WAB, B_VVVV, N * v, v, v, v, (int)(v * vv), (int)vv, v, 1,
                                   (int)(v * vv), (int)vv, v, 1, offD, offS))) return rc;
            }
            {   // + sum_r t_r^b(kb) ovvv[kb,ka,ke](r,a,e,f)
                GemmSpec s; s.a = B_OVVV; s.b = B_T1; s.c = B_WAB;
                s.M = (int)(vv * v); s.N = v; s.K = o; s.nbatch = (int)(p1 - p0) * N; s.nchunk = 1;
                for (size_t p = p0; p < p1; ++p) for (int ke = 0; ke < N; ++ke) {
                    const int ka = pairs[p].first, kb = pairs[p].second;
                    s.offA.push_back(blk(Sovvv, kb, ka, ke)); s.offB.push_back(kb * ov);
                    s.offC.push_back(((long long)(p - p0) * N + ke) * Svvvv);
                }
                s.rowA = tab({{(int)(vv * v), 1}}); s.colA = tab({{o, vv * v}});
                s.rowB = tab({{o, v}}); s.colB = tab({{v, 1}});
                s.rowC = tab({{v, vv * v}, {(int)vv, 1}}); s.colC = tab({{v, vv}});
                if ((rc = G(s))) return rc;
            }
            {   // - sum_r t_r^a(ka) ovvv[ka,kb,ke](r,b,e,f)
                GemmSpec s; s.a = B_OVVV; s.b = B_T1; s.c = B_WAB; s.ar = -1.0;
                s.M = (int)(vv * v); s.N = v; s.K = o; s.nbatch = (int)(p1 - p0) * N; s.nchunk = 1;
                for (size_t p = p0; p < p1; ++p) for (int ke = 0; ke < N; ++ke) {
                    const int ka = pairs[p].first, kb = pairs[p].second;
                    s.offA.push_back(blk(Sovvv, ka, kb, ke)); s.offB.push_back(ka * ov);
                    s.offC.push_back(((long long)(p - p0) * N + ke) * Svvvv);
                }
                s.rowA = tab({{(int)(vv * v), 1}}); s.colA = tab({{o, vv * v}});
                s.rowB = tab({{o, v}}); s.colB = tab({{v, 1}});
                s.rowC = tab({{v, vv}, {(int)vv, 1}}); s.colC = tab({{v, vv * v}});
                if ((rc = G(s))) return rc;
            }
            h->cur_name = "ladder";
            // R2 += 1/2 sum_{ke,e,f} tau_ij^ef W'^abef, packed by antisymmetry: tau and W'
            // change sign under (e ke) <-> (f kf), so the half sum over ordered pairs is the
            // full sum over (ke < kf, all e f) plus (ke = kf, e < f); W' also changes sign
            // under (a ka) <-> (b kb), so only (ka < kb, all a b) and (ka = kb, a < b) are
            // computed and the mirror R2(ba) = -R2(ab) is written by the same thread.  Four
            // launches per slab: {ka < kb, ka = kb} x {ke < kf, ke = kf}.
            for (int diag_ab = 0; diag_ab < 2; ++diag_ab) {
                for (int diag_ef = 0; diag_ef < 2; ++diag_ef) {
                    GemmSpec s; s.a = B_TAU; s.b = B_WAB; s.c = B_R2; s.ar = 1.0;
                    const std::vector<int>& ncols = diag_ab ? pairs_lt : pairs_full;
                    const std::vector<int>& kcols = diag_ef ? pairs_lt : pairs_full;
                    s.M = (int)oo; s.N = (int)ncols.size(); s.K = (int)kcols.size(); s.nchunk = N;
                    s.nbatch = 0;
                    for (size_t p = p0; p < p1; ++p) {
                        const int ka = pairs[p].first, kb = pairs[p].second;
                        if ((ka == kb) != (diag_ab == 1)) continue;
                        const int S = kg.k4(ka, kb, 0);
                        std::vector<int> kes;
                        for (int ke = 0; ke < N; ++ke) {
                            const int kf = kg.k4(S, 0, ke);
                            if (diag_ef ? (ke == kf) : (ke < kf)) kes.push_back(ke);
                        }
                        if (kes.empty() || (v < 2 && (diag_ab || diag_ef))) continue;
                        for (int ki = 0; ki < N; ++ki) {
                            const int kj = kg.k4(ka, kb, ki);
                            for (int c = 0; c < N; ++c) {
                                const int ke = kes[std::min<size_t>(c, kes.size() - 1)];
                                s.offA.push_back(blk(S2, ki, kj, ke));
                                s.offB.push_back(((long long)(p - p0) * N + ke) * Svvvv);
                            }
                            s.nchunk_b.push_back((int)kes.size());
                            s.offC.push_back(blk(S2, ki, kj, ka));
                            s.offC2.push_back(blk(S2, ki, kj, kb));
                            ++s.nbatch;
                        }
                    }
                    if (s.nbatch == 0) { if ((rc = G(s))) return rc; continue; }
                    s.rowA = tab({{(int)oo, vv}}); s.colA = kcols;
                    s.rowB = kcols; s.colB.clear();
                    for (int x : ncols) s.colB.push_back(x * (int)vv);
                    s.rowC = tab({{(int)oo, vv}}); s.colC = ncols;
                    s.colC2.clear();
                    // the mirror of (a, b) is (b, a): in block kb for ka < kb, in the same
                    // block for ka = kb
                    for (int x : ncols) s.colC2.push_back(swapped[x]);
                    if ((rc = G(s))) return rc;
                }
            }
            // the tensor-core path forms W' inside its operand embedding
            if (tcp) for (size_t i = w_first; i < h->seq.size(); ++i) h->seq[i].mode = 1;
        }
    }
    for (TcSet& T : sets) {
        h->cur_oz = T.oz;
        // Tensor-core ladder, antisymmetry-packed like the FP64 one: outputs (ka < kb | ka = kb,
        // a < b) with the mirror R2(ba) = -R2(ab), contractions over (ke < kf | ke = kf, e < f).
        // A' = tau rows [S = ki + kj][ke][ki](ij), columns the (e f) list; B' = W' formed
        // straight into its embedding for the blocks of one chunk at a time (the buffer
        // holds T.lb_floats per part), each chunk followed by its GEMM.
        std::vector<long long> so_lad;
        for (int S = 0; S < N; ++S) for (int ke = 0; ke < N; ++ke) for (int ki = 0; ki < N; ++ki)
            so_lad.push_back(blk(S2, ki, kg.k4(S, 0, ki), ke));
        std::vector<int> full_vv = tab({{(int)vv, 1}}), lt_vv;
        for (int x = 0; x < v; ++x) for (int y = x + 1; y < v; ++y) lt_vv.push_back(x * v + y);
        const int M = (int)(N * oo);
        for (int diag_ef = 0; diag_ef < 2; ++diag_ef) {
            const std::vector<int>& efl = diag_ef ? lt_vv : full_vv;
            if (efl.empty()) continue;
            const TcBuf& A = diag_ef ? T.lap : T.la;
            if ((rc = add_embed(h, al, B_TAU, A, 0, (int)oo, (int)efl.size(), so_lad, tab({{(int)oo, vv}}), efl, false)))
                return rc;
            for (int diag_ab = 0; diag_ab < 2; ++diag_ab) {
                const std::vector<int>& abl = diag_ab ? lt_vv : full_vv;
                if (abl.empty()) continue;
                std::vector<std::pair<int, int>> batches;
                std::vector<std::vector<int>> chunks;
                for (int ka = 0; ka < N; ++ka) for (int kb = ka; kb < N; ++kb) {
                    if ((ka == kb) != (diag_ab == 1)) continue;
                    const int S = kg.k4(ka, kb, 0);
                    std::vector<int> kes;
                    for (int ke = 0; ke < N; ++ke) { const int kf = kg.k4(S, 0, ke); if (diag_ef ? ke == kf : ke < kf) kes.push_back(ke); }
                    if (kes.empty()) continue;
                    batches.push_back({ka, kb});
                    chunks.push_back(kes);
                }
                const long long rows_per_block = 2LL * (long long)abl.size();
                const long long cap_rows = T.lb_floats / A.kpad;
                size_t b0 = 0;
                while (b0 < batches.size()) {
                    // as many (ka, kb) batches as their W' blocks fit in the buffer (at least one)
                    size_t b1 = b0;
                    long long rows = 0;
                    while (b1 < batches.size() && (b1 == b0 || rows + (long long)chunks[b1].size() * rows_per_block <= cap_rows)) {
                        rows += (long long)chunks[b1].size() * rows_per_block;
                        ++b1;
                    }
                    if (rows > cap_rows) return CCSD_ERR_INVALID;
                    TcBuf B{T.lb.big, T.lb.big + T.lb_floats, std::max(rows, 1LL), A.kpad};
                    if (!pooled) B.small = T.lb.small;
                    if (T.oz) { B.big = B.small = nullptr; B.sl = T.lb.sl; B.sc = T.lb.sc; }
                    int nchmax = 0;
                    for (size_t bb = b0; bb < b1; ++bb) nchmax = std::max<int>(nchmax, (int)chunks[bb].size());
                    std::vector<int> blk3, ra, rb, cc, cc2, cnt;
                    std::vector<long long> oc, oc2;
                    int used = 0;
                    for (size_t bb = b0; bb < b1; ++bb) {
                        const int ka = batches[bb].first, kb = batches[bb].second;
                        const int S = kg.k4(ka, kb, 0);
                        const std::vector<int>& kes = chunks[bb];
                        for (int c = 0; c < nchmax; ++c) {
                            const int cc_ = std::min<int>(c, (int)kes.size() - 1);
                            ra.push_back((int)((((long long)S * N + kes[cc_]) * N) * oo));
                            rb.push_back((int)((long long)(used + cc_) * rows_per_block));
                        }
                        for (int ke : kes) { blk3.push_back(ka); blk3.push_back(kb); blk3.push_back(ke); }
                        used += (int)kes.size();
                        cnt.push_back((int)kes.size());
                        for (int ki = 0; ki < N; ++ki)
                            for (int ij = 0; ij < (int)oo; ++ij) {
                                oc.push_back(blk(S2, ki, kg.k4(S, 0, ki), ka) + ij * vv);
                                oc2.push_back(blk(S2, ki, kg.k4(S, 0, ki), kb) + ij * vv);
                            }
                    }
                    WListPlan wl{};
                    wl.a.big = B.big; wl.a.small = B.small;
                    wl.a.blk = upload(al, blk3, h->st);
                    wl.a.abl = upload(al, abl, h->st);
                    wl.a.efl = upload(al, efl, h->st);
                    if (al.err) return al.err;
                    {   // groups of consecutive pairs with the same a (the list is ordered by a)
                        std::vector<int> grp;
                        for (int x = 0; x < (int)abl.size();) {
                            int y = x + 1;
                            while (y < (int)abl.size() && y - x < WP_GROUP && abl[y] / v == abl[x] / v) ++y;
                            grp.push_back(x); grp.push_back(y - x);
                            x = y;
                        }
                        wl.a.grp = upload(al, grp, h->st);
                        if (al.err) return al.err;
                        wl.a.ngrp = (int)(grp.size() / 2);
                    }
                    wl.a.nblk = (int)(blk3.size() / 3); wl.a.nab = (int)abl.size(); wl.a.nef = (int)efl.size();
                    wl.a.N = N; wl.a.o = o; wl.a.v = v; wl.a.Kpad = A.kpad;
                    if (T.oz) {
                        wl.oz = true;
                        OzWprimeArgs& z = wl.z;
                        z.sl = B.sl; z.sc = B.sc; z.rows = B.rows;
                        z.blk = wl.a.blk; z.abl = wl.a.abl; z.efl = wl.a.efl;
                        z.nblk = wl.a.nblk; z.nab = wl.a.nab; z.nef = wl.a.nef;
                        z.N = N; z.o = o; z.v = v; z.Kpad = A.kpad; z.slices = h->oz_slices;
                    }
                    h->wlists.push_back(wl);
                    Step st{10, (int)h->wlists.size() - 1, "ladder_W", 0.0, 40.0 * (double)wl.a.nblk * wl.a.nab * wl.a.nef};
                    st.mode = tc_mode(h);
                    h->seq.push_back(st);
                    cc.clear(); cc2.clear();
                    for (int x : abl) { cc.push_back(x); cc2.push_back((x % v) * v + x / v); }
                    if ((rc = add_tc(h, al, A, B, B_R2, M, (int)(2 * abl.size()), (int)(b1 - b0), nchmax, ra, rb, oc, cc,
                                     1.0, 3, cnt, oc2, cc2))) return rc;
                    b0 = b1;
                }
            }
        }
    }
    h->cur_name = "ring_W_t1";
    // ring: W~_jn^bf (Eq. Def_Woovv), stored [kj,kn,kb](j,n,b,f), kf = kn + kb - kj
    {
        std::vector<long long> offD, offS;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            const int kf = kg.k4(kn, kb, kj);
            offD.push_back(blk(S2, kj, kn, kb)); offS.push_back(blk(S2, kn, kb, kf));
        }
        // W(j,n,b,f) = ovvo(n,b,f,j)
        if ((rc = add_perm(h, al, B_WRING, B_OVVO, o, o, v, v, (int)(o * vv), (int)vv, v, 1,
                           1, (int)(vv * o), (int)(v * o), o, offD, offS))) return rc;
    }
    {   // + sum_c t_j^c <n b||f c>
        GemmSpec s; s.a = B_T1; s.b = B_OVVV; s.c = B_WRING;
        s.M = o; s.N = (int)(o * vv); s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            const int kf = kg.k4(kn, kb, kj);
            s.offA.push_back(kj * ov); s.offB.push_back(blk(Sovvv, kn, kb, kf)); s.offC.push_back(blk(S2, kj, kn, kb));
        }
        s.rowA = tab({{o, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{(int)(o * vv), v}});
        s.rowC = tab({{o, o * vv}}); s.colC = tab({{(int)(o * vv), 1}});
        if ((rc = G(s))) return rc;
    }
    {   // Q(n,r,j,f) = ooov[kn,kb,kj](n,r,j,f) - sum_c oovv[kn,kb,kf](n,r,f,c) t_j^c
        std::vector<long long> offD, offS;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            offD.push_back(blk(Sooov, kj, kn, kb)); offS.push_back(blk(Sooov, kn, kb, kj));
        }
        if ((rc = add_perm(h, al, B_Q, B_OOOV, o, o, o, v, (int)(oo * v), (int)ov, v, 1,
                           (int)(oo * v), (int)ov, v, 1, offD, offS))) return rc;
        GemmSpec s; s.a = B_OOVV; s.b = B_T1; s.c = B_Q; s.ar = -1.0;
        s.M = (int)(oo * v); s.N = o; s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            const int kf = kg.k4(kn, kb, kj);
            s.offA.push_back(blk(S2, kn, kb, kf)); s.offB.push_back(kj * ov); s.offC.push_back(blk(Sooov, kj, kn, kb));
        }
        s.rowA = tab({{(int)oo, vv}, {v, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{(int)oo, ov}, {v, 1}}); s.colC = tab({{o, v}});
        if ((rc = G(s))) return rc;
    }
    {   // W += sum_r t_r^b Q(n,r,j,f)   (= -t_r^b <n r||f j> - t_j^c t_r^b <n r||f c>)
        GemmSpec s; s.a = B_T1; s.b = B_Q; s.c = B_WRING;
        s.M = v; s.N = (int)(oo * v); s.K = o; s.nbatch = N3; s.nchunk = 1;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            s.offA.push_back(kb * ov); s.offB.push_back(blk(Sooov, kj, kn, kb)); s.offC.push_back(blk(S2, kj, kn, kb));
        }
        s.rowA = tab({{v, 1}}); s.colA = tab({{o, v}});
        s.rowB = tab({{o, ov}}); s.colB = tab({{o, oo * v}, {o, v}, {v, 1}});
        s.rowC = tab({{v, v}}); s.colC = tab({{o, vv}, {o, o * vv}, {v, 1}});
        if ((rc = G(s))) return rc;
    }
    h->cur_name = "ring_W_t2";
    {   // W -= 1/2 sum_kx t_{j x}^{y b} <n x||f y>
        GemmSpec s; s.a = B_T2; s.b = B_OOVV; s.c = B_WRING; s.ar = -0.5;
        s.M = (int)ov; s.N = (int)ov; s.K = (int)ov; s.nbatch = N3; s.nchunk = N;
        for (int kj = 0; kj < N; ++kj) for (int kn = 0; kn < N; ++kn) for (int kb = 0; kb < N; ++kb) {
            const int kf = kg.k4(kn, kb, kj);
            for (int kx = 0; kx < N; ++kx) {
                const int ky = kg.k4(kj, kx, kb);
                s.offA.push_back(blk(S2, kj, kx, ky)); s.offB.push_back(blk(S2, kn, kx, kf));
            }
            s.offC.push_back(blk(S2, kj, kn, kb));
        }
        s.rowA = tab({{o, o * vv}, {v, 1}}); s.colA = tab({{o, vv}, {v, v}});
        s.rowB = tab({{o, vv}, {v, 1}}); s.colB = tab({{o, o * vv}, {v, v}});
        s.rowC = tab({{o, o * vv}, {v, v}}); s.colC = tab({{o, vv}, {v, 1}});
        if ((rc = G(s))) return rc;
        if (tcp) h->seq.back().mode = 1;
    }
    for (TcSet& T : sets) {
        h->cur_oz = T.oz;
        // Both ring GEMMs on tensor cores, one batch per momentum transfer D:
        //   ring W:  rows (kj, j, b) with kb = kj - D, columns (kn, n, f) with kf = kn - D
        //   ring C:  rows (ki, i, a) with ka = ki - D, columns (kj, j, b) with kb = kj + D
        // so every output row and column of a batch is a full momentum block and the
        // output offset stays separable (row part + column part).  A' rows are
        // [D][chunk][first](first index, second index) of t2[first, chunk, second] with
        // second = first - D; since t_jx^yb = -t_jx^by it serves both GEMMs (the sign
        // of the W term is folded into alpha).
        std::vector<long long> so;
        for (int D = 0; D < N; ++D) for (int kc = 0; kc < N; ++kc) for (int kf_ = 0; kf_ < N; ++kf_)
            so.push_back(blk(S2, kf_, kc, kg.k4(kf_, 0, D)));
        if ((rc = add_embed(h, al, B_T2, T.ra, 0, (int)ov, (int)ov, so, tab({{o, o * vv}, {v, v}}),
                            tab({{o, vv}, {v, 1}}), false))) return rc;
        // B of ring W: <n kn x kx||f kf y ky> rows (n,f), columns (x,y): [D][kx][kn], kf = kn - D
        so.clear();
        for (int D = 0; D < N; ++D) for (int kx = 0; kx < N; ++kx) for (int kn = 0; kn < N; ++kn)
            so.push_back(blk(S2, kn, kx, kg.k4(kn, 0, D)));
        if ((rc = add_embed(h, al, B_OOVV, T.b1, 1, (int)ov, (int)ov, so, tab({{o, o * vv}, {v, v}}),
                            tab({{o, vv}, {v, 1}}), !pooled))) return rc;
        std::vector<int> ra, rb, cc; std::vector<long long> oc;
        for (int D = 0; D < N; ++D) {
            for (int kx = 0; kx < N; ++kx) {
                ra.push_back((int)(((long long)D * N + kx) * N * ov));
                rb.push_back((int)(((long long)D * N + kx) * N * 2 * ov));
            }
            for (int kj = 0; kj < N; ++kj) {
                const int kb = kg.k4(kj, 0, D);
                for (int j = 0; j < o; ++j) for (int b = 0; b < v; ++b)
                    oc.push_back(((long long)kj * N * N + kb) * S2 + j * o * vv + b * v);
            }
        }
        for (int kn = 0; kn < N; ++kn) for (int n = 0; n < o; ++n) for (int f = 0; f < v; ++f)
            cc.push_back((int)((long long)kn * N * S2 + n * vv + f));
        if ((rc = add_tc(h, al, T.ra, T.b1, B_WRING, (int)(N * ov), (int)(2 * N * ov), N, N, ra, rb, oc, cc, 0.5, 3)))
            return rc;
    }
    h->cur_name = "ring";
    {   // ZR = sum_kn t_{in}^{af} W_{jn}^{bf}
        GemmSpec s; s.a = B_T2; s.b = B_WRING; s.c = B_ZR; s.acc = false;
        s.M = (int)ov; s.N = (int)ov; s.K = (int)ov; s.nbatch = N3; s.nchunk = N;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            const int kb = kg.k4(ki, kj, ka);
            for (int kn = 0; kn < N; ++kn) { s.offA.push_back(blk(S2, ki, kn, ka)); s.offB.push_back(blk(S2, kj, kn, kb)); }
            s.offC.push_back(blk(S2, ki, kj, ka));
        }
        s.rowA = tab({{o, o * vv}, {v, v}}); s.colA = tab({{o, vv}, {v, 1}});
        s.rowB = tab({{o, vv}, {v, 1}}); s.colB = tab({{o, o * vv}, {v, v}});
        s.rowC = tab({{o, o * vv}, {v, v}}); s.colC = tab({{o, vv}, {v, 1}});
        if ((rc = G(s))) return rc;
        if (tcp) h->seq.back().mode = 1;
    }
    for (TcSet& T : sets) {
        h->cur_oz = T.oz;
        add_zero(h, B_ZR);
        // B_ring[D][kn][kj]: rows (j,b), columns (n,f) of W~[kj, kn, kb], kb = kj + D
        std::vector<long long> so;
        for (int D = 0; D < N; ++D) for (int kn = 0; kn < N; ++kn) for (int kj = 0; kj < N; ++kj)
            so.push_back(blk(S2, kj, kn, kg.k4(kj, D, 0)));
        if ((rc = add_embed(h, al, B_WRING, T.rb, 1, (int)ov, (int)ov, so, tab({{o, o * vv}, {v, v}}),
                            tab({{o, vv}, {v, 1}}), false))) return rc;
        std::vector<int> ra, rb, cc; std::vector<long long> oc;
        for (int D = 0; D < N; ++D) {
            for (int kn = 0; kn < N; ++kn) {
                ra.push_back((int)(((long long)D * N + kn) * N * ov));
                rb.push_back((int)(((long long)D * N + kn) * N * 2 * ov));
            }
            for (int ki = 0; ki < N; ++ki) {
                const int ka = kg.k4(ki, 0, D);
                for (int i2 = 0; i2 < o; ++i2) for (int a = 0; a < v; ++a)
                    oc.push_back(((long long)ki * N * N + ka) * S2 + i2 * o * vv + a * v);
            }
        }
        for (int kj = 0; kj < N; ++kj) for (int j = 0; j < o; ++j) for (int b = 0; b < v; ++b)
            cc.push_back((int)((long long)kj * N * S2 + j * vv + b));
        if ((rc = add_tc(h, al, T.ra, T.rb, B_ZR, (int)(N * ov), (int)(2 * N * ov), N, N, ra, rb, oc, cc, 1.0, 3)))
            return rc;
    }
    h->cur_name = "ring_t1t1";
    {   // TT(r,b,i,j) = sum_c <r ka b kb||c ki j kj> t_i^c ;  ZR -= sum_r t_r^a TT(r,b,i,j)
        GemmSpec s; s.a = B_OVVO; s.b = B_T1; s.c = B_TT; s.acc = false;
        s.M = (int)(ov * o); s.N = o; s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            const int kb = kg.k4(ki, kj, ka);
            s.offA.push_back(blk(S2, ka, kb, ki)); s.offB.push_back(ki * ov); s.offC.push_back(blk(Sooov, ki, kj, ka));
        }
        s.rowA = tab({{(int)ov, v * o}, {o, 1}}); s.colA = tab({{v, o}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{o, v}});
        s.rowC = tab({{(int)ov, oo}, {o, 1}}); s.colC = tab({{o, o}});
        if ((rc = G(s))) return rc;
        GemmSpec s2; s2.a = B_T1; s2.b = B_TT; s2.c = B_ZR; s2.ar = -1.0;
        s2.M = v; s2.N = (int)(oo * v); s2.K = o; s2.nbatch = N3; s2.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            s2.offA.push_back(ka * ov); s2.offB.push_back(blk(Sooov, ki, kj, ka)); s2.offC.push_back(blk(S2, ki, kj, ka));
        }
        s2.rowA = tab({{v, 1}}); s2.colA = tab({{o, v}});
        s2.rowB = tab({{o, v * oo}}); s2.colB = tab({{(int)oo, 1}, {v, oo}});
        s2.rowC = tab({{v, v}}); s2.colC = tab({{(int)oo, vv}, {v, 1}});
        if ((rc = G(s2))) return rc;
    }
    h->cur_name = "fock_t1_terms";
    const size_t fock_first = h->seq.size();
    // remaining terms under P(ab) and P(ij)
    // The P(ab)-only terms (call them Zab) and the P(ij)-only terms (Zij) accumulate into
    // ZR at half weight: Zab is antisymmetric in (i,j) and Zij in (a,b), so
    // P(ij)P(ab) (Zab/2) = P(ab) Zab and P(ij)P(ab) (Zij/2) = P(ij) Zij, and one permuted
    // sum finishes all of R2's terms.
    {   // ZR += 1/2 sum_f t_ij^af F'^{bf}(kb)
        GemmSpec s; s.a = B_T2; s.b = B_FVVP; s.c = B_ZR; s.ar = 0.5;
        s.M = (int)(oo * v); s.N = v; s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            const int kb = kg.k4(ki, kj, ka);
            s.offA.push_back(blk(S2, ki, kj, ka)); s.offB.push_back(kb * vv); s.offC.push_back(blk(S2, ki, kj, ka));
        }
        s.rowA = tab({{(int)(oo * v), v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, 1}}); s.colB = tab({{v, v}});
        s.rowC = tab({{(int)(oo * v), v}}); s.colC = tab({{v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // ZR -= 1/2 sum_r t_r^a <r b||i j> = 1/2 sum_r t_r^a conj(ooov[ki,kj,ka](i,j,r,b))
        GemmSpec s; s.a = B_T1; s.b = B_OOOV; s.c = B_ZR; s.ar = -0.5; s.conjB = true;
        s.M = v; s.N = (int)(oo * v); s.K = o; s.nbatch = N3; s.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            s.offA.push_back(ka * ov); s.offB.push_back(blk(Sooov, ki, kj, ka)); s.offC.push_back(blk(S2, ki, kj, ka));
        }
        s.rowA = tab({{v, 1}}); s.colA = tab({{o, v}});
        s.rowB = tab({{o, v}}); s.colB = tab({{(int)oo, ov}, {v, 1}});
        s.rowC = tab({{v, v}}); s.colC = tab({{(int)oo, vv}, {v, 1}});
        if ((rc = G(s))) return rc;
    }
    {   // ZR -= 1/2 sum_n t_{i n}^{ab} F'_{nj}(kj)
        GemmSpec s; s.a = B_T2; s.b = B_FOOP; s.c = B_ZR; s.ar = -0.5;
        s.M = (int)(o * vv); s.N = o; s.K = o; s.nbatch = N3; s.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            s.offA.push_back(blk(S2, ki, kj, ka)); s.offB.push_back(kj * oo); s.offC.push_back(blk(S2, ki, kj, ka));
        }
        s.rowA = tab({{o, o * vv}, {(int)vv, 1}}); s.colA = tab({{o, vv}});
        s.rowB = tab({{o, o}}); s.colB = tab({{o, 1}});
        s.rowC = tab({{o, o * vv}, {(int)vv, 1}}); s.colC = tab({{o, vv}});
        if ((rc = G(s))) return rc;
    }
    {   // ZR += 1/2 sum_c <a b||c j> t_i^c = - 1/2 sum_c t_i^c conj(ovvv[kj,ki,ka](j,c,a,b))
        GemmSpec s; s.a = B_T1; s.b = B_OVVV; s.c = B_ZR; s.ar = -0.5; s.conjB = true;
        s.M = o; s.N = (int)(o * vv); s.K = v; s.nbatch = N3; s.nchunk = 1;
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka) {
            s.offA.push_back(ki * ov); s.offB.push_back(blk(Sovvv, kj, ki, ka)); s.offC.push_back(blk(S2, ki, kj, ka));
        }
        s.rowA = tab({{o, v}}); s.colA = tab({{v, 1}});
        s.rowB = tab({{v, vv}}); s.colB = tab({{o, vv * v}, {(int)vv, 1}});
        s.rowC = tab({{o, o * vv}}); s.colC = tab({{o, vv}, {(int)vv, 1}});
        if ((rc = G(s))) return rc;
    }
    if (mixed) {
        // the four GEMMs above run outside mixed iterations only; mixed iterations fuse them
        for (size_t i = fock_first; i < h->seq.size(); ++i) h->seq[i].mode = 4;
        h->shadow[B_FVVP] = (float2*)al.get((size_t)h->bufsize[B_FVVP] * 8);
        h->shadow[B_FOOP] = (float2*)al.get((size_t)h->bufsize[B_FOOP] * 8);
        if (al.err) return al.err;
        Step s1{12, B_FVVP, h->cur_name, 0.0, 24.0 * h->bufsize[B_FVVP]};
        Step s2{9, B_FOOP, h->cur_name, 0.0, 24.0 * h->bufsize[B_FOOP]};
        Step s3{11, 0, h->cur_name, 8.0 * 2.0 * (o + v) * (double)h->n2, 8.0 * 4.0 * h->n2};
        s1.mode = s2.mode = s3.mode = 3;
        h->seq.push_back(s1); h->seq.push_back(s2); h->seq.push_back(s3);
    }
    if (h->has_oz) {
        // Ozaki iterations: the four GEMMs above become one fused double-float pass
        // (fock_terms_df_kernel) over double-float copies; the GEMMs stay for FP64 iterations
        for (size_t i = fock_first; i < h->seq.size(); ++i)
            if (h->seq[i].kind == 0) h->seq[i].mode = 1;
        if (!h->in32[B_OOOV]) {
            h->ooov_df = (df2*)al.get((size_t)h->bufsize[B_OOOV] * sizeof(df2));
            if (al.err) return al.err;
            if (!al.dry)
                to_df2_kernel<<<ew_grid(h->bufsize[B_OOOV]), 256, 0, h->st>>>(h->ooov_df, h->buf[B_OOOV],
                                                                             h->bufsize[B_OOOV]);
        }
        if (pooled && pool_b_bytes >= (long long)sizeof(df2) * h->n2) {
            h->t2_df = (df2*)pool_b;          // idle between the last tensor-core GEMM and the next residual
        } else {
            h->t2_df = (df2*)al.get((size_t)h->n2 * sizeof(df2));
        }
        h->t1_df = (df2*)al.get((size_t)h->n1 * sizeof(df2));
        h->fvvpT_df = (df2*)al.get((size_t)h->bufsize[B_FVVP] * sizeof(df2));
        h->foop_df = (df2*)al.get((size_t)h->bufsize[B_FOOP] * sizeof(df2));
        if (al.err) return al.err;
        Step s1{14, 0, h->cur_name, 0.0, 32.0 * (double)(h->n2 + h->n1)};
        Step s2{13, 0, h->cur_name, 8.0 * 2.0 * (o + v) * (double)h->n2, 16.0 * 4.0 * h->n2};
        s1.mode = s2.mode = 5;
        h->seq.push_back(s1); h->seq.push_back(s2);
    }
    h->seq.push_back({4, 0, "antisym_R2", 0.0, 16.0 * 3.0 * h->n2});
    h->cur_oz = true;
    if (oz && (rc = oz_convert_gemms(h, al, oz_specs, pooled, pool_a, pool_b, pool_ae, pool_be, pool_asc, pool_bsc,
                                     pool_ar, pool_br)))
        return rc;
    return 0;
}


void set_sizes(ccsd_ctx* h) {
    const long long N = h->N, o = h->o, v = h->v, N3 = N * N * N;
    const long long sz[NBUF] = {N * o * o, N * v * v, N * o * v, N3 * o * o * o * o, N3 * o * o * o * v,
                                N3 * o * o * v * v, N3 * o * o * v * v, N3 * o * v * v * v, N3 * v * v * v * v,
                                h->n1, h->n2, h->n1, h->n2, h->n2, h->n2,
                                N * o * v, N * o * o, N * v * v, N * o * o, N * v * v,
                                N3 * o * o * o * o, wab_pairs_per_slab(N, v, h->wab_cap_bytes) * N * v * v * v * v,
                                h->n2, N3 * o * o * o * v, N3 * o * o * o * v,
                                h->n2, h->n2, h->n2};
    for (int i = 0; i < NBUF; ++i) h->bufsize[i] = sz[i];
}

// One CTA per row for the row-wise operand kernels (grid-stride beyond 2^31 - 1 rows).
dim3 row_grid(long long rows) {
    return dim3((unsigned)std::max(1LL, std::min(rows, 2147483647LL)));
}

dim3 ew_grid(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    if (b < 1) b = 1;
    return dim3((unsigned)b);
}

int launch_gemm(ccsd_ctx* h, GemmPlan& p) {
    if (p.blocks == 0) return 0;
    GemmArgs g = h->fp32 ? p.args32 : p.args;
    g.A = h->buf[p.a]; g.B = h->buf[p.b]; g.C = h->buf[p.c]; g.work = h->work;
    g.A32 = (h->fp32 || h->in32[p.a]) ? h->shadow[p.a] : nullptr;
    g.B32 = (h->fp32 || h->in32[p.b]) ? h->shadow[p.b] : nullptr;
    dim3 grid((unsigned)p.blocks, (unsigned)g.nsplit);
    // the K-split tile shapes pay off in FP32 only (measured on GB300: the double-float
    // instance ran slower with them, the FP64 one no faster); the other instances take
    // the plain shape with the same tile, so the plan's tiling and split-K stand
    const int cfg = h->fp32 ? p.cfg : p.cfg == CFG_16x16K ? CFG_16x16 : p.cfg == CFG_32x16K ? CFG_32x16 : p.cfg;
    if (h->oz_on) {         // Ozaki form: the GEMMs left off the tensor cores run in double-float
        switch (cfg) {
            case CFG_64x64:  zgemm_kb_kernel<64, 64, 8, 4, 4, df><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_64x32:  zgemm_kb_kernel<64, 32, 8, 4, 2, df><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_128x16: zgemm_kb_kernel<128, 16, 8, 8, 1, df><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16:  zgemm_kb_kernel<32, 16, 8, 2, 1, df><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16K: zgemm_kb_kernel<32, 16, 32, 2, 2, df, 2><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_16x16K: zgemm_kb_kernel<16, 16, 32, 2, 2, df, 4><<<grid, 256, 0, h->st>>>(g); break;
            default:         zgemm_kb_kernel<16, 16, 8, 1, 1, df><<<grid, 256, 0, h->st>>>(g); break;
        }
    } else if (h->fp32) {
        switch (cfg) {
            case CFG_64x64:  zgemm_kb_kernel<64, 64, 8, 4, 4, float><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_64x32:  zgemm_kb_kernel<64, 32, 8, 4, 2, float><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_128x16: zgemm_kb_kernel<128, 16, 8, 8, 1, float><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16:  zgemm_kb_kernel<32, 16, 8, 2, 1, float><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16K: zgemm_kb_kernel<32, 16, 32, 2, 2, float, 2><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_16x16K: zgemm_kb_kernel<16, 16, 32, 2, 2, float, 4><<<grid, 256, 0, h->st>>>(g); break;
            default:         zgemm_kb_kernel<16, 16, 8, 1, 1, float><<<grid, 256, 0, h->st>>>(g); break;
        }
    } else {
        switch (cfg) {
            case CFG_64x64:  zgemm_kb_kernel<64, 64, 8, 4, 4><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_64x32:  zgemm_kb_kernel<64, 32, 8, 4, 2><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_128x16: zgemm_kb_kernel<128, 16, 8, 8, 1><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16:  zgemm_kb_kernel<32, 16, 8, 2, 1><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_32x16K: zgemm_kb_kernel<32, 16, 32, 2, 2, double, 2><<<grid, 256, 0, h->st>>>(g); break;
            case CFG_16x16K: zgemm_kb_kernel<16, 16, 32, 2, 2, double, 4><<<grid, 256, 0, h->st>>>(g); break;
            default:         zgemm_kb_kernel<16, 16, 8, 1, 1><<<grid, 256, 0, h->st>>>(g); break;
        }
    }
    ++h->launches;
    if (g.nsplit > 1) {
        zgemm_split_reduce<<<ew_grid((long long)g.nbatch * g.M * g.N), 256, 0, h->st>>>(g);
        ++h->launches;
    }
    return 0;
}

// Kernel arguments of plan steps, with the handle's buffers resolved.
CopyOp copy_op(const ccsd_ctx* h, const CopyPlan& c) {
    return CopyOp{h->buf[c.dst], h->in32[c.src] ? nullptr : h->buf[c.src], h->in32[c.src] ? h->shadow[c.src] : nullptr,
                  c.n, c.conj};
}

PermOp perm_op(const ccsd_ctx* h, const PermPlan& pp) {
    return PermOp{h->buf[pp.dst], h->in32[pp.src] ? nullptr : h->buf[pp.src],
                  h->in32[pp.src] ? h->shadow[pp.src] : nullptr, pp.p};
}

TauOp tau_op(const ccsd_ctx* h) {
    const bool c64 = h->fp32 && h->cfg.precision == CCSD_MIXED;
    return TauOp{h->buf[B_T1], h->buf[B_T2], h->buf[B_TAU], h->buf[B_TAUT], h->kb_of, h->N, h->o, h->v,
                 c64 ? h->shadow[B_T2] : nullptr, c64 ? h->shadow[B_TAUT] : nullptr};
}

FockTermsOp fock_terms_op(const ccsd_ctx* h) {
    return FockTermsOp{h->buf[B_ZR], h->shadow[B_T2], h->shadow[B_T1], h->shadow[B_FVVP], h->shadow[B_FOOP],
                       h->shadow[B_OOOV], h->shadow[B_OVVV], h->kb_of, h->N, h->o, h->v};
}

WprimeListArgs wprime_op(const ccsd_ctx* h, const WListPlan& w) {
    WprimeListArgs a = w.a;
    a.vvvv = h->shadow[B_VVVV];
    a.ovvv = h->shadow[B_OVVV]; a.t1 = h->shadow[B_T1];
    return a;
}

// The tiled W' kernel serves o <= WPT_OMAX and v <= 128 (its t1 tables in shared memory).
bool wprime_tiled(const WprimeListArgs& a) { return a.o <= WPT_OMAX && a.v <= 128; }

EmbedArgs embed_op(const ccsd_ctx* h, const EmbedPlan& e) {
    EmbedArgs a = e.a;
    a.src = h->buf[e.src];
    a.src32 = h->in32[e.src] ? h->shadow[e.src] : nullptr;
    return a;
}

UpdateOp update_op(const ccsd_ctx* h, const int* skip) {
    return UpdateOp{h->buf[B_T1], h->buf[B_T2], h->buf[B_R1], h->buf[B_R2], h->eo, h->ev, h->kb_of,
                    h->N, h->o, h->v, nullptr, nullptr, skip};
}

void launch_embed(ccsd_ctx* h, EmbedPlan& e) {
    if (e.oz) {
        OzEmbedArgs z = e.z;
        z.src = h->buf[e.src];
        z.src32 = h->in32[e.src] ? h->shadow[e.src] : nullptr;
        const long long rows = (long long)z.nblk * z.R;
        if (z.Kpad / 2 <= 64)       // one warp per row
            oz_embed_kernel<<<row_grid((rows + 7) / 8), 256, 0, h->st>>>(z);
        else
            oz_embed_kernel<<<row_grid(rows), z.Kpad / 2 >= 256 ? 256 : 128, 0, h->st>>>(z);
        ++h->launches;
        return;
    }
    const EmbedArgs a = embed_op(h, e);
    embed_kernel<<<row_grid((long long)a.nblk * a.R), a.Kpad / 2 >= 256 ? 256 : 128, 0, h->st>>>(a);
    ++h->launches;
}

// A kernel's dynamic shared-memory limit is an attribute of the current device: it
// is raised once per device and kernel, under a lock (the serving loop launches from
// its own thread).
enum { SMEM_TC = 0, SMEM_OZ = 1, SMEM_OZ_WPRIME = 2, SMEM_TC_GROUPED = 3 };
std::mutex g_smem_attr_mu;
std::set<std::pair<int, int>> g_smem_attr_done;

void ensure_smem_attr(int which) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
    std::lock_guard<std::mutex> lock(g_smem_attr_mu);
    if (!g_smem_attr_done.insert(std::make_pair(dev, which)).second) return;
    switch (which) {
        case SMEM_TC:
            cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
            break;
        case SMEM_OZ:
            cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
            break;
        case SMEM_TC_GROUPED:
            cudaFuncSetAttribute(tc_gemm_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
            break;
        default:
            cudaFuncSetAttribute(oz_wprime_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            break;
    }
}

void launch_tc(ccsd_ctx* h, TcPlan& t) {
    if (t.oz) {
        ensure_smem_attr(SMEM_OZ);
        OzArgs z = t.z;
        z.C = h->buf[t.c];
        z.work = z.nsplit > 1 ? h->oz_work : nullptr;
        oz_gemm_kernel<<<t.blocks, OZ_THREADS, OZ_SMEM_BYTES, h->st>>>(t.mA_big, t.mB_big, z);
        ++h->launches;
        if (z.work) {
            oz_split_reduce<<<ew_grid((long long)z.nbatch * z.M * (z.Nr / 2)), 256, 0, h->st>>>(z);
            ++h->launches;
        }
        return;
    }
    ensure_smem_attr(SMEM_TC);
    TcArgs a = t.a;
    a.C = h->buf[t.c];
    tc_gemm_kernel<<<t.blocks, TC_THREADS, TC_SMEM_BYTES, h->st>>>(t.mA_big, t.mA_small, t.mB_big, t.mB_small, a);
    ++h->launches;
}

// Accumulate the elapsed time of traced steps [a, b) (synchronizes the stream).
bool step_active(const ccsd_ctx* h, const Step& s);

int trace_collect(ccsd_ctx* h, size_t a, size_t b) {
    CK(cudaStreamSynchronize(h->st));
    for (size_t i = a; i < b; ++i) {
        if (i < h->seq.size() && !step_active(h, h->seq[i])) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev0[i], h->ev1[i]));
        h->step_ms[i] += ms;
        h->step_calls[i] += 1;
    }
    return 0;
}

bool step_active(const ccsd_ctx* h, const Step& s) {
    const bool mixed_it = h->fp32 && h->cfg.precision == CCSD_MIXED;   // a mixed (FP32) iteration
    const bool tc = mixed_it || h->oz_on;                              // tensor-core contractions
    switch (s.mode) {
        case 1: return !tc;
        case 2: return mixed_it;
        case 3: return mixed_it;
        case 4: return !mixed_it;
        case 5: return h->oz_on != 0;
        default: return true;
    }
}

// Launches plan step si (no tracing, no mode check).
void launch_step(ccsd_ctx* h, size_t si) {
    const int N = h->N, o = h->o, v = h->v;
    const Step& s = h->seq[si];
        switch (s.kind) {
            case 0: launch_gemm(h, h->gemms[s.idx]); break;
            case 1: {
                const CopyPlan& c = h->copies[s.idx];
                copy_kernel<<<ew_grid(c.n), 256, 0, h->st>>>(copy_op(h, c));
                ++h->launches;
                break;
            }
            case 2: {
                const PermPlan& pp = h->perms[s.idx];
                const dim3 g = ew_grid((long long)pp.p.nbatch * pp.p.n0 * pp.p.n1 * pp.p.n2 * pp.p.n3);
                permute4_kernel<<<g, 256, 0, h->st>>>(perm_op(h, pp));
                ++h->launches;
                break;
            }
            case 3:
                tau_kernel<<<ew_grid(h->n2), 256, 0, h->st>>>(tau_op(h));
                ++h->launches;
                break;
            case 4:
                antisym_kernel<<<ew_grid(h->n2), 256, 0, h->st>>>(AntisymOp{h->buf[B_R2], h->buf[B_ZR], h->kb_of, N, o, v});
                ++h->launches;
                break;
            case 5: launch_embed(h, h->embeds[s.idx]); break;
            case 6: launch_tc(h, h->tcs[s.idx]); break;
            case 7:
                cudaMemsetAsync(h->buf[s.idx], 0, (size_t)h->bufsize[s.idx] * 16, h->st);
                break;
            case 10: {
                if (h->wlists[s.idx].oz) {
                    ensure_smem_attr(SMEM_OZ_WPRIME);
                    OzWprimeArgs z = h->wlists[s.idx].z;
                    if (h->in32[B_VVVV]) { z.vvvv32 = h->shadow[B_VVVV]; z.vvvv = nullptr; }
                    else { z.vvvv = h->buf[B_VVVV]; z.vvvv32 = nullptr; }
                    if (h->in32[B_OVVV]) { z.ovvv32 = h->shadow[B_OVVV]; z.ovvv_df = nullptr; }
                    else { z.ovvv_df = h->ovvv_df; z.ovvv32 = nullptr; }
                    z.t1 = h->buf[B_T1];
                    oz_wprime_kernel<<<row_grid((long long)z.nblk * z.nab), 256, (size_t)(z.nef + 2 * z.o) * 16,
                                       h->st>>>(z);
                    ++h->launches;
                    break;
                }
                const WprimeListArgs a = wprime_op(h, h->wlists[s.idx]);
                if (wprime_tiled(a)) {
                    const WprimeTileOp op{a, a.nab != a.v * a.v ? 1 : 0};
                    wprime_tile_kernel<<<row_grid((long long)a.nblk * ((a.v + WPT_A - 1) / WPT_A)), 256, 0, h->st>>>(op);
                } else {
                    wprime_list_kernel<<<row_grid((long long)a.nblk * a.ngrp), 256, 0, h->st>>>(a);
                }
                ++h->launches;
                break;
            }
            case 11: {   // mixed form: fused P(ab)-only / P(ij)-only terms into ZR
                fock_terms_kernel<<<ew_grid(h->n2), 256, 0, h->st>>>(fock_terms_op(h));
                ++h->launches;
                break;
            }
            case 13:  // Ozaki iterations: fused double-float Fock terms into ZR
                fock_terms_df_kernel<<<ew_grid(h->n2), 256, 0, h->st>>>(FockTermsDfOp{
                    h->buf[B_ZR], h->t2_df, h->t1_df, h->fvvpT_df, h->foop_df,
                    h->ooov_df, h->in32[B_OOOV] ? h->shadow[B_OOOV] : nullptr,
                    h->ovvv_df, h->in32[B_OVVV] ? h->shadow[B_OVVV] : nullptr, h->kb_of, N, o, v});
                ++h->launches;
                break;
            case 14:  // their double-float copies
                to_df_kernel<<<ew_grid(h->n2 + h->n1), 256, 0, h->st>>>(ToDfOp{
                    h->t2_df, h->buf[B_T2], h->n2, h->t1_df, h->buf[B_T1], h->n1,
                    h->fvvpT_df, h->buf[B_FVVP], h->foop_df, h->buf[B_FOOP], N, o, v});
                ++h->launches;
                break;
            case 12:  // complex64 copy of F'vv, transposed per k (fused Fock terms)
                to_c64_transpose_kernel<<<ew_grid(h->bufsize[s.idx]), 256, 0, h->st>>>(ToC64TOp{h->shadow[s.idx], h->buf[s.idx], N, v});
                ++h->launches;
                break;
            case 9:   // refresh the complex64 copy of an amplitude or intermediate buffer
                to_c64_kernel<<<ew_grid(h->bufsize[s.idx]), 256, 0, h->st>>>(ToC64Op{h->shadow[s.idx], h->buf[s.idx], h->bufsize[s.idx]});
                ++h->launches;
                break;
        }
}

// Enqueues one residual evaluation; no host synchronization.
int run_residual_async(ccsd_ctx* h) {
    for (size_t si = 0; si < h->seq.size(); ++si) {
        if (!step_active(h, h->seq[si])) continue;
        if (h->trace) cudaEventRecord(h->ev0[si], h->st);
        launch_step(h, si);
        if (h->trace) cudaEventRecord(h->ev1[si], h->st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { last_err(e); return CCSD_ERR_CUDA; }
    return 0;
}

// A bounded wait inside a tensor-core GEMM gave up: report, clear, fail (synchronizes).
int check_tc_err(ccsd_ctx* h) {
    if (!((h->fp32 && h->cfg.precision == CCSD_MIXED) || h->oz_on) || !h->tc_err) return 0;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (flag) {
        snprintf(g_errbuf, sizeof g_errbuf, "tensor-core GEMM wait timed out (code %d)", flag);
        CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->st));
        return CCSD_ERR_TIMEOUT;
    }
    return 0;
}

int run_residual(ccsd_ctx* h) {
    int rc = run_residual_async(h);
    if (rc) return rc;
    if ((rc = check_tc_err(h))) return rc;
    if (h->trace) return trace_collect(h, 0, h->seq.size());
    return 0;
}


// ================================================================ grouped iterations
// Many independent problems advance together (the batched form, the serving loop).
// Problems whose plans have the same step sequence (kinds and modes; sizes differ)
// form a group, and every step of one iteration is ONE launch over all members of
// the group:
//   * contractions: zgemm_grouped_kernel, a persistent CTA set striding a
//     [member][split][batch][tile] work list, with one tile shape per step (picked by
//     an autotuner in the batched form); split-K reductions grouped the same way;
//   * tensor-core contractions: tc_gemm_grouped_kernel, one CTA per tile of every
//     member, each member's tensor maps and arguments read from global memory;
//   * elementwise and row-wise steps (tau, copies, permutations, operand embedding,
//     W' formation, Fock terms, antisymmetrization, zeroing): grouped_op_kernel;
//   * max|R| per member, and the update of the members not yet converged.
// The group's launch descriptors are built once per membership on the host.
struct BatchGroup {
    int cfg = CFG_64x64;
    std::vector<GemmArgs> args;       // per member, tiles for `cfg`, pointers resolved
    GemmArgs* d_args = nullptr;
    long long* d_prefix = nullptr;
    long long total = 0;
    std::vector<int> split_members;
    std::function<void(cudaStream_t)> reduce;   // grouped split-K reduction (members that split)
};

// One grouped launch: enqueues itself on a stream (no host synchronization).
struct GLaunch {
    std::function<void(cudaStream_t)> fn;
    int launches = 0;
    int gemm = -1;                    // index into Group::gemms for contraction steps
};

struct Group {
    std::vector<ccsd_ctx*> m;
    std::vector<int> ids;             // caller's member indices (batched form)
    std::vector<uint64_t> rids;       // request ids of the members (serving form): a handle's
                                      // address can be reused by a later request, an id is not
    int fp32 = 0;
    std::vector<size_t> steps;        // active plan steps, the same in every member
    std::vector<GLaunch> res;         // the residual, in plan order
    std::vector<BatchGroup> gemms;
    GLaunch norms, update;
    double* d_norms = nullptr;        // max|R| of each member (a caller's slice, or owned)
    int* d_skip = nullptr;            // serving form: per member, 1 = no update this round
    int* d_err = nullptr;             // shared error word of the grouped tensor-core launches
    std::vector<void*> owned;         // device allocations of this group
    struct ChunkPool* pool = nullptr; // chunks for the tables (null: allocated per group)
    std::vector<void*> chunks;        // chunks taken from the pool
    char* chunk = nullptr;
    size_t chunk_used = 0;
};

// Step signature of a plan: members with equal signatures share every grouped launch.
std::vector<std::pair<int, int>> plan_signature(const ccsd_ctx* h) {
    std::vector<std::pair<int, int>> sig;
    for (const Step& st : h->seq) sig.emplace_back(st.kind, st.mode);
    return sig;
}

// Device memory of a group's tables: 256-byte aligned pieces of 4 MiB chunks.  A
// serving loop rebuilds groups whenever its admitted solves change, so the chunks
// come from a pool that outlives the groups (no cudaMalloc or cudaFree per rebuild).
constexpr size_t kChunkBytes = 4u << 20;

struct ChunkPool {
    std::vector<void*> free_chunks, all;
    ~ChunkPool() { for (void* p : all) cudaFree(p); }
    void* get() {
        if (!free_chunks.empty()) { void* p = free_chunks.back(); free_chunks.pop_back(); return p; }
        void* p = nullptr;
        if (cudaMalloc(&p, kChunkBytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        all.push_back(p);
        return p;
    }
};

int group_alloc(Group& G, size_t bytes, void** p) {
    bytes = (std::max<size_t>(bytes, 16) + 255) / 256 * 256;
    if (bytes > kChunkBytes) {            // a table larger than a chunk: its own allocation
        if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_OOM; }
        G.owned.push_back(*p);
        return 0;
    }
    if (!G.chunk || G.chunk_used + bytes > kChunkBytes) {
        void* c = G.pool ? G.pool->get() : nullptr;
        if (!G.pool) {
            if (cudaMalloc(&c, kChunkBytes) != cudaSuccess) { cudaGetLastError(); c = nullptr; }
            else G.owned.push_back(c);
        } else if (c) {
            G.chunks.push_back(c);
        }
        if (!c) return CCSD_ERR_OOM;
        G.chunk = (char*)c;
        G.chunk_used = 0;
    }
    *p = G.chunk + G.chunk_used;
    G.chunk_used += bytes;
    return 0;
}

template <class T>
T* group_upload(Group& G, const std::vector<T>& v, cudaStream_t st, int* rc) {
    void* p = nullptr;
    if ((*rc = group_alloc(G, v.size() * sizeof(T), &p))) return nullptr;
    if (cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        *rc = CCSD_ERR_CUDA;
        return nullptr;
    }
    return (T*)p;
}

void group_free(Group& G) {
    for (void* p : G.owned) cudaFree(p);
    if (G.pool) for (void* c : G.chunks) G.pool->free_chunks.push_back(c);
    ChunkPool* pool = G.pool;
    G = Group();
    G.pool = pool;
}

long long grid_blocks(const dim3& g) { return (long long)g.x; }
// row-wise ops stride their rows: a member's share of a grouped launch is bounded
long long row_blocks(long long rows) { return std::max(1LL, std::min(rows, 8192LL)); }

// A grouped launch of one operation type over the members; blocks[i] = member i's grid.
template <class Op>
int make_grouped(Group& G, const std::vector<Op>& ops, const std::vector<long long>& blocks, cudaStream_t st,
                 GLaunch& out) {
    std::vector<long long> prefix(1, 0);
    for (long long b : blocks) prefix.push_back(prefix.back() + b);
    const long long total = prefix.back();
    if (total > 2147483647LL) { refuse("a grouped launch exceeds 2^31 - 1 blocks"); return CCSD_ERR_INVALID; }
    int rc = 0;
    const Op* d_ops = group_upload(G, ops, st, &rc);
    if (rc) return rc;
    const long long* d_prefix = group_upload(G, prefix, st, &rc);
    if (rc) return rc;
    const int n = (int)ops.size();
    out.launches = total > 0 ? 1 : 0;
    out.fn = [d_ops, d_prefix, n, total](cudaStream_t s) {
        if (total > 0) grouped_op_kernel<Op><<<(unsigned)total, 256, 0, s>>>(d_ops, d_prefix, n);
    };
    return 0;
}

long long tiles_for(const GemmArgs& a, int cfg, int* tm, int* tn) {
    *tm = (a.M + CFG_BM[cfg] - 1) / CFG_BM[cfg];
    *tn = (a.N + CFG_BN[cfg] - 1) / CFG_BN[cfg];
    return (long long)*tm * *tn * a.nbatch;
}

int group_gemm_descriptors(Group& G, BatchGroup& bg, size_t si, int cfg, cudaStream_t st, bool own_split = false) {
    const int n = (int)G.m.size();
    bg.cfg = cfg;
    bg.args.clear();
    bg.split_members.clear();
    // Split-K by load balance: the persistent CTAs stride one work list, so no work item
    // (a tile and its share of the chunks) should hold more than half the mean load of a
    // CTA.  Skinny contractions (a few tiles over a long K, like the F~ and R1 sums) are
    // then spread over many CTAs even when the whole group has plenty of tiles.
    double total_work = 0.0;             // sum over members of tiles x K x chunks
    for (int i = 0; i < n; ++i) {
        int tm, tn;
        const GemmArgs& a0 = G.m[i]->gemms[G.m[i]->seq[si].idx].args;
        total_work += (double)tiles_for(a0, cfg, &tm, &tn) * a0.K * a0.nchunk;
    }
    const double item_cap = std::max(1.0, 0.5 * total_work / (double)(kSMs * 8));
    long long tot = 0;
    std::vector<long long> prefix;
    std::vector<SplitReduceOp> red;
    std::vector<long long> red_blocks;
    for (int i = 0; i < n; ++i) {
        ccsd_ctx* h = G.m[i];
        const GemmPlan& p = h->gemms[h->seq[si].idx];
        GemmArgs a = G.fp32 ? p.args32 : p.args;
        int tm, tn;
        tiles_for(a, cfg, &tm, &tn);
        if (own_split) {
            if (cfg != p.cfg) { refuse("members of a split-keeping group must share each step's tile shape"); return CCSD_ERR_INVALID; }
            a.A = h->buf[p.a]; a.B = h->buf[p.b]; a.C = h->buf[p.c]; a.work = h->work;
            a.A32 = (G.fp32 || h->in32[p.a]) ? h->shadow[p.a] : nullptr;
            a.B32 = (G.fp32 || h->in32[p.b]) ? h->shadow[p.b] : nullptr;
            if (a.nsplit > 1) {
                bg.split_members.push_back(i);
                red.push_back(SplitReduceOp{a});
                red_blocks.push_back(grid_blocks(ew_grid((long long)a.nbatch * a.M * a.N)));
            }
            prefix.push_back(tot);
            tot += (long long)tm * tn * a.nbatch * a.nsplit;
            bg.args.push_back(a);
            continue;
        }
        a.tiles_m = tm; a.tiles_n = tn;
        const int ns = std::max(1, std::min(a.nchunk, (int)std::ceil((double)a.K * a.nchunk / item_cap)));
        a.chunks_per_split = (a.nchunk + ns - 1) / ns;
        a.nsplit = (a.nchunk + a.chunks_per_split - 1) / a.chunks_per_split;
        if (G.fp32) {        // the FP32 instance keeps its partial sums short (see finalize_gemm)
            const GemmArgs& g32 = p.args32;
            if (g32.chunks_per_split < a.chunks_per_split) {
                a.chunks_per_split = g32.chunks_per_split;
                a.nsplit = (a.nchunk + a.chunks_per_split - 1) / a.chunks_per_split;
            }
        }
        if (a.nbatch == 0) a.nsplit = 1;
        if (a.nsplit > 1) {
            const size_t need = (size_t)a.nsplit * a.nbatch * a.M * a.N;
            if (need > h->work_elems) {          // the handle owns its split-K workspace
                void* w = nullptr;
                if (cudaMalloc(&w, need * 16) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_OOM; }
                h->owned.push_back(w);
                h->owned_bytes += need * 16;
                h->work = (double2*)w;
                h->work_elems = need;
            }
            bg.split_members.push_back(i);
        }
        a.A = h->buf[p.a]; a.B = h->buf[p.b]; a.C = h->buf[p.c]; a.work = h->work;
        a.A32 = (G.fp32 || h->in32[p.a]) ? h->shadow[p.a] : nullptr;
        a.B32 = (G.fp32 || h->in32[p.b]) ? h->shadow[p.b] : nullptr;
        prefix.push_back(tot);
        tot += (long long)tm * tn * a.nbatch * a.nsplit;
        bg.args.push_back(a);
        if (a.nsplit > 1) {
            red.push_back(SplitReduceOp{a});
            red_blocks.push_back(grid_blocks(ew_grid((long long)a.nbatch * a.M * a.N)));
        }
    }
    prefix.push_back(tot);
    bg.total = tot;
    if (!bg.d_args) {
        void* x = nullptr;
        int rc = group_alloc(G, sizeof(GemmArgs) * n, &x);
        if (rc) return rc;
        bg.d_args = (GemmArgs*)x;
        if ((rc = group_alloc(G, sizeof(long long) * (n + 1), &x))) return rc;
        bg.d_prefix = (long long*)x;
    }
    CK(cudaMemcpyAsync(bg.d_args, bg.args.data(), sizeof(GemmArgs) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(bg.d_prefix, prefix.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st));
    bg.reduce = nullptr;
    if (!red.empty()) {
        GLaunch gl;
        int rc = make_grouped(G, red, red_blocks, st, gl);
        if (rc) return rc;
        bg.reduce = gl.fn;
    }
    return 0;
}

template <int BM, int BN, int BK, int TM, int TN, int KS = 1>
void grouped_gemm_launch(const BatchGroup& bg, int fp32, cudaStream_t st, int n) {
    const long long ctas = std::min<long long>(bg.total, (long long)kSMs * 8);
    if (fp32)
        zgemm_grouped_kernel<BM, BN, BK, TM, TN, float, KS><<<(unsigned)ctas, 256, 0, st>>>(bg.d_args, bg.d_prefix, n, bg.total);
    else
        zgemm_grouped_kernel<BM, BN, BK, TM, TN, double, KS><<<(unsigned)ctas, 256, 0, st>>>(bg.d_args, bg.d_prefix, n, bg.total);
}

void launch_gemm_group(const BatchGroup& bg, int fp32, cudaStream_t st, int n) {
    if (bg.total <= 0 || !bg.d_args) return;
    const int cfg = fp32 ? bg.cfg : bg.cfg == CFG_16x16K ? CFG_16x16 : bg.cfg == CFG_32x16K ? CFG_32x16 : bg.cfg;
    switch (cfg) {
        case CFG_64x64: grouped_gemm_launch<64, 64, 8, 4, 4>(bg, fp32, st, n); break;
        case CFG_64x32: grouped_gemm_launch<64, 32, 8, 4, 2>(bg, fp32, st, n); break;
        case CFG_128x16: grouped_gemm_launch<128, 16, 8, 8, 1>(bg, fp32, st, n); break;
        case CFG_32x16: grouped_gemm_launch<32, 16, 8, 2, 1>(bg, fp32, st, n); break;
        case CFG_32x16K: grouped_gemm_launch<32, 16, 32, 2, 2, 2>(bg, fp32, st, n); break;
        case CFG_16x16K: grouped_gemm_launch<16, 16, 32, 2, 2, 4>(bg, fp32, st, n); break;
        default: grouped_gemm_launch<16, 16, 8, 1, 1>(bg, fp32, st, n); break;
    }
    if (bg.reduce) bg.reduce(st);
}

// Builds every grouped launch of one iteration of the group's members.  d_norms[i]
// receives member i's max|R| (null: the group allocates its own array); d_skip[i] != 0
// skips its update (may be null: all update).  cfgs: tile shape of each contraction
// step (empty: each step's own shape in member 0).  own_split: every member keeps the
// split-K choice of its own plan (its results are then bitwise those of a plain
// iteration; the members must share each step's tile shape).
int group_build(Group& G, int fp32, const std::vector<int>& cfgs, double* d_norms, const int* d_skip,
                cudaStream_t st, bool own_split = false) {
    const int n = (int)G.m.size();
    if (n == 0) return 0;
    G.fp32 = fp32;
    ccsd_ctx* h0 = G.m[0];
    int rc = group_alloc(G, sizeof(int), (void**)&G.d_err);
    if (rc) return rc;
    if (!d_norms && (rc = group_alloc(G, sizeof(double) * n, (void**)&d_norms))) return rc;
    G.d_norms = d_norms;
    CK(cudaMemsetAsync(G.d_err, 0, sizeof(int), st));
    G.steps.clear();
    for (size_t si = 0; si < h0->seq.size(); ++si)
        if (step_active(h0, h0->seq[si])) G.steps.push_back(si);
    int ngemm = 0;
    for (size_t si : G.steps) if (h0->seq[si].kind == 0) ++ngemm;
    G.gemms.assign(ngemm, BatchGroup());
    int gi = 0;
    ensure_smem_attr(SMEM_TC_GROUPED);
    for (size_t si : G.steps) {
        const Step& s0 = h0->seq[si];
        GLaunch gl;
        switch (s0.kind) {
            case 0: {
                const int cfg = gi < (int)cfgs.size() ? cfgs[gi] : h0->gemms[s0.idx].cfg;
                if ((rc = group_gemm_descriptors(G, G.gemms[gi], si, cfg, st, own_split))) return rc;
                const BatchGroup* bg = &G.gemms[gi];
                gl.gemm = gi;
                gl.launches = (bg->total > 0 ? 1 : 0) + (bg->reduce ? 1 : 0);
                gl.fn = [bg, fp32, n](cudaStream_t s) { launch_gemm_group(*bg, fp32, s, n); };
                ++gi;
                break;
            }
            case 1: case 2: case 3: case 4: case 7: case 9: case 11: case 12: {
                // elementwise steps
                std::vector<long long> blocks;
                auto build = [&](auto make, auto count) {
                    using Op = decltype(make(G.m[0]));
                    std::vector<Op> ops;
                    for (ccsd_ctx* h : G.m) { ops.push_back(make(h)); blocks.push_back(grid_blocks(ew_grid(count(h)))); }
                    return make_grouped(G, ops, blocks, st, gl);
                };
                if (s0.kind == 1)
                    rc = build([&](ccsd_ctx* h) { return copy_op(h, h->copies[h->seq[si].idx]); },
                               [&](ccsd_ctx* h) { return h->copies[h->seq[si].idx].n; });
                else if (s0.kind == 2)
                    rc = build([&](ccsd_ctx* h) { return perm_op(h, h->perms[h->seq[si].idx]); },
                               [&](ccsd_ctx* h) {
                                   const Perm4& q = h->perms[h->seq[si].idx].p;
                                   return (long long)q.nbatch * q.n0 * q.n1 * q.n2 * q.n3;
                               });
                else if (s0.kind == 3)
                    rc = build([&](ccsd_ctx* h) { return tau_op(h); }, [&](ccsd_ctx* h) { return h->n2; });
                else if (s0.kind == 4)
                    rc = build([&](ccsd_ctx* h) { return AntisymOp{h->buf[B_R2], h->buf[B_ZR], h->kb_of, h->N, h->o, h->v}; },
                               [&](ccsd_ctx* h) { return h->n2; });
                else if (s0.kind == 7)
                    rc = build([&](ccsd_ctx* h) { return ZeroOp{h->buf[h->seq[si].idx], h->bufsize[h->seq[si].idx]}; },
                               [&](ccsd_ctx* h) { return h->bufsize[h->seq[si].idx]; });
                else if (s0.kind == 9)
                    rc = build([&](ccsd_ctx* h) {
                                   const int bi = h->seq[si].idx;
                                   return ToC64Op{h->shadow[bi], h->buf[bi], h->bufsize[bi]};
                               },
                               [&](ccsd_ctx* h) { return h->bufsize[h->seq[si].idx]; });
                else if (s0.kind == 11)
                    rc = build([&](ccsd_ctx* h) { return fock_terms_op(h); }, [&](ccsd_ctx* h) { return h->n2; });
                else
                    rc = build([&](ccsd_ctx* h) {
                                   const int bi = h->seq[si].idx;
                                   return ToC64TOp{h->shadow[bi], h->buf[bi], h->N, h->v};
                               },
                               [&](ccsd_ctx* h) { return h->bufsize[h->seq[si].idx]; });
                if (rc) return rc;
                break;
            }
            case 5: {
                std::vector<EmbedArgs> ops;
                std::vector<long long> blocks;
                for (ccsd_ctx* h : G.m) {
                    const EmbedPlan& e = h->embeds[h->seq[si].idx];
                    if (e.oz) { refuse("grouped launches run split-TF32 and FP64 steps only"); return CCSD_ERR_INVALID; }
                    ops.push_back(embed_op(h, e));
                    blocks.push_back(row_blocks((long long)e.a.nblk * e.a.R));
                }
                if ((rc = make_grouped(G, ops, blocks, st, gl))) return rc;
                break;
            }
            case 10: {
                std::vector<WprimeListArgs> ops;
                std::vector<WprimeTileOp> tops;
                std::vector<long long> blocks, tblocks;
                bool tiled = true;
                for (ccsd_ctx* h : G.m) {
                    const WListPlan& w = h->wlists[h->seq[si].idx];
                    if (w.oz) { refuse("grouped launches run split-TF32 and FP64 steps only"); return CCSD_ERR_INVALID; }
                    const WprimeListArgs a = wprime_op(h, w);
                    ops.push_back(a);
                    blocks.push_back(row_blocks((long long)a.nblk * a.ngrp));
                    tops.push_back(WprimeTileOp{a, a.nab != a.v * a.v ? 1 : 0});
                    tblocks.push_back(row_blocks((long long)a.nblk * ((a.v + WPT_A - 1) / WPT_A)));
                    tiled = tiled && wprime_tiled(a);
                }
                if ((rc = tiled ? make_grouped(G, tops, tblocks, st, gl) : make_grouped(G, ops, blocks, st, gl))) return rc;
                break;
            }
            case 6: {
                std::vector<CUtensorMap> maps;
                std::vector<TcArgs> args;
                std::vector<long long> prefix(1, 0);
                for (ccsd_ctx* h : G.m) {
                    const TcPlan& t = h->tcs[h->seq[si].idx];
                    if (t.oz) { refuse("grouped launches run split-TF32 and FP64 steps only"); return CCSD_ERR_INVALID; }
                    maps.push_back(t.mA_big); maps.push_back(t.mA_small);
                    maps.push_back(t.mB_big); maps.push_back(t.mB_small);
                    TcArgs a = t.a;
                    a.C = h->buf[t.c];
                    a.err = G.d_err;
                    args.push_back(a);
                    prefix.push_back(prefix.back() + t.blocks);
                }
                const long long total = prefix.back();
                if (total > 2147483647LL) { refuse("a grouped launch exceeds 2^31 - 1 blocks"); return CCSD_ERR_INVALID; }
                const CUtensorMap* d_maps = group_upload(G, maps, st, &rc);
                if (rc) return rc;
                const TcArgs* d_args = group_upload(G, args, st, &rc);
                if (rc) return rc;
                const long long* d_prefix = group_upload(G, prefix, st, &rc);
                if (rc) return rc;
                gl.launches = total > 0 ? 1 : 0;
                gl.fn = [d_maps, d_args, d_prefix, n, total](cudaStream_t s) {
                    if (total > 0)
                        tc_gemm_grouped_kernel<<<(unsigned)total, TC_THREADS, TC_SMEM_BYTES, s>>>(d_maps, d_args, d_prefix, n);
                };
                break;
            }
            default:
                refuse("a plan step kind has no grouped launch");
                return CCSD_ERR_INVALID;
        }
        G.res.push_back(gl);
    }
    // max|R| of every member, then the update of those not converged
    {
        std::vector<MaxabsOp> mx;
        std::vector<FinalMaxOp> fm;
        std::vector<UpdateOp> up;
        std::vector<long long> bm, bf, bu;
        for (int i = 0; i < n; ++i) {
            ccsd_ctx* h = G.m[i];
            const long long nn = h->n1 + h->n2;
            mx.push_back(MaxabsOp{h->res, nn, h->red});
            bm.push_back(h->red_blocks);
            fm.push_back(FinalMaxOp{h->red, h->red_blocks, d_norms + i});
            bf.push_back(1);
            up.push_back(update_op(h, d_skip ? d_skip + i : nullptr));
            bu.push_back(grid_blocks(ew_grid(nn)));
        }
        GLaunch a1, a2;
        if ((rc = make_grouped(G, mx, bm, st, a1)) || (rc = make_grouped(G, fm, bf, st, a2)))
            return rc;
        G.norms.launches = a1.launches + a2.launches;
        G.norms.fn = [a1, a2](cudaStream_t s) { a1.fn(s); a2.fn(s); };
        const int depth = h0->cfg.diis_depth;
        for (ccsd_ctx* h : G.m)
            if (h->cfg.diis_depth != depth) { refuse("the members of a group share one DIIS depth"); return CCSD_ERR_INVALID; }
        if (depth == 0) {
            if ((rc = make_grouped(G, up, bu, st, G.update))) return rc;
        } else {
            // DIIS on the device, on each member's own history (the handle's DIIS state):
            // pack, inner products, Pulay solve, extrapolation -- the kernels and grids of
            // ccsd_iterate, so a member's iterates are those it has alone
            std::vector<DiisPackOp> pk;
            std::vector<DiisDotOp> dt;
            std::vector<DiisSolveOp> sv;
            std::vector<DiisComboOp> cb;
            std::vector<long long> bp, bd, bs, bc;
            for (int i = 0; i < n; ++i) {
                ccsd_ctx* h = G.m[i];
                if (!h->d_diis) { refuse("a group member has no DIIS state"); return CCSD_ERR_INVALID; }
                const int* skip = d_skip ? d_skip + i : nullptr;
                const long long blk = (long long)h->o * h->o * h->v * h->v;
                pk.push_back(DiisPackOp{h->amp, h->res, h->d_diis, h->d_cblk, h->nc, h->d_rden, h->N, h->o, h->v,
                                        skip});
                bp.push_back(grid_blocks(ew_grid(h->n1 + h->nc * blk)));
                dt.push_back(DiisDotOp{h->d_diis, h->n1, blk, h->nc, h->d_cw, h->d_diis_part, h->red_blocks, skip});
                bd.push_back(h->red_blocks);
                sv.push_back(DiisSolveOp{h->d_diis, h->d_diis_part, h->red_blocks, skip});
                bs.push_back(1);
                cb.push_back(DiisComboOp{h->amp, h->d_diis, h->d_ctgt, h->nc, h->N, h->o, h->v, skip});
                bc.push_back(std::min<long long>(cb.back().units(), 8LL * kSMs));
            }
            GLaunch g1, g2, g3, g4;
            if ((rc = make_grouped(G, pk, bp, st, g1)) || (rc = make_grouped(G, dt, bd, st, g2)) ||
                (rc = make_grouped(G, sv, bs, st, g3)) || (rc = make_grouped(G, cb, bc, st, g4)))
                return rc;
            G.update.launches = g1.launches + g2.launches + g3.launches + g4.launches;
            G.update.fn = [g1, g2, g3, g4](cudaStream_t s) { g1.fn(s); g2.fn(s); g3.fn(s); g4.fn(s); };
        }
    }
    CK(cudaStreamSynchronize(st));
    return 0;
}

void group_residual(const Group& G, cudaStream_t st) {
    for (const GLaunch& gl : G.res) gl.fn(st);
}

int group_launches(const Group& G, bool with_update) {
    int n = G.norms.launches + (with_update ? G.update.launches : 0);
    for (const GLaunch& gl : G.res) n += gl.launches;
    return n;
}

// Reads and clears the group's tensor-core error word (synchronizes st).
int group_check_err(const Group& G, cudaStream_t st) {
    if (!G.d_err) return 0;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, G.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) {
        snprintf(g_errbuf, sizeof g_errbuf, "tensor-core GEMM wait timed out (code %d)", flag);
        CK(cudaMemsetAsync(G.d_err, 0, sizeof(int), st));
        return CCSD_ERR_TIMEOUT;
    }
    return 0;
}

}  // namespace

// ================================================================ batched form
// n independent problems: members are partitioned into groups by plan signature;
// one iteration (every group's residual, max|R| per member, update of the members
// not converged) is captured once in a CUDA graph, each group on a stream of its own
// (they run concurrently), and replayed.
struct ccsd_batch {
    int n = 0;
    std::vector<ccsd_ctx*> m;
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> gst;                 // one stream per group
    std::vector<cudaEvent_t> gev;
    int fp32 = 0;
    std::vector<std::unique_ptr<Group>> groups;   // held by pointer: launches keep pointers into them
    int tuned = 0;
    std::vector<void*> owned;
    double* d_norms = nullptr;
    int* d_done = nullptr;
    std::vector<int> done;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t fork = nullptr;
};

namespace {

int batch_alloc(ccsd_batch* B, size_t bytes, void** p) {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_OOM; }
    B->owned.push_back(*p);
    return 0;
}

// Residual of every member, max|R| into d_norms, update of unconverged members; the
// groups run on their own streams, forked from and joined into B->st.
void batch_iteration_body(ccsd_batch* B) {
    cudaEventRecord(B->fork, B->st);
    for (size_t g = 0; g < B->groups.size(); ++g) {
        cudaStreamWaitEvent(B->gst[g], B->fork, 0);
        group_residual(*B->groups[g], B->gst[g]);
        B->groups[g]->norms.fn(B->gst[g]);
        B->groups[g]->update.fn(B->gst[g]);
        cudaEventRecord(B->gev[g], B->gst[g]);
        cudaStreamWaitEvent(B->st, B->gev[g], 0);
    }
}

// Autotuner: times every tile shape on every grouped contraction and keeps the
// fastest.  Safe at any time: each residual re-initializes what it accumulates.
int batch_autotune(ccsd_batch* B) {
    const int cands[CFG_COUNT] = {CFG_64x64, CFG_64x32, CFG_128x16, CFG_32x16, CFG_16x16, CFG_32x16K, CFG_16x16K};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = 0;
    for (auto& gp : B->groups) {
        Group& G = *gp;
        const int n = (int)G.m.size();
        size_t gi = 0;
        for (size_t k = 0; k < G.res.size() && !rc; ++k) {
            if (G.res[k].gemm < 0) continue;
            BatchGroup& bg = G.gemms[G.res[k].gemm];
            const size_t si = G.steps[k];
            int best = bg.cfg;
            float best_ms = 1e30f;
            for (int c : cands) {
                if ((rc = group_gemm_descriptors(G, bg, si, c, B->st))) break;
                launch_gemm_group(bg, B->fp32, B->st, n);     // warm
                cudaEventRecord(e0, B->st);
                launch_gemm_group(bg, B->fp32, B->st, n);
                cudaEventRecord(e1, B->st);
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    last_err(cudaGetLastError());
                    rc = CCSD_ERR_CUDA;
                    break;
                }
                if (ms < best_ms) { best_ms = ms; best = c; }
            }
            if (!rc) rc = group_gemm_descriptors(G, bg, si, best, B->st);
            G.res[k].launches = (bg.total > 0 ? 1 : 0) + (bg.reduce ? 1 : 0);
            ++gi;
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    CK(cudaStreamSynchronize(B->st));
    B->tuned = 1;
    return 0;
}

int batch_capture(ccsd_batch* B) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal));
    batch_iteration_body(B);
    cudaError_t e = cudaStreamEndCapture(B->st, &g);
    if (e != cudaSuccess) { last_err(e); return CCSD_ERR_CUDA; }
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { last_err(e); return CCSD_ERR_CUDA; }
    return 0;
}

bool valid_cfg(const ccsd_config* c) {
    if (!c) return refuse("config is null");
    for (int i = 0; i < 3; ++i) if (c->nk_dims[i] < 1 || c->nk_dims[i] > 64) return refuse("nk_dims must be 1..64");
    if (c->nocc < 1 || c->nvir < 1 || c->nocc > 256 || c->nvir > 512) return refuse("nocc must be 1..256, nvir 1..512");
    if (c->precision != CCSD_FP64 && c->precision != CCSD_MIXED && c->precision != CCSD_OZAKI)
        return refuse("unknown precision");
    if (c->precision == CCSD_MIXED && (c->polish_iters < 0 || c->polish_iters > 100))
        return refuse("polish_iters must be 0..100");
    if (c->polish_precision != CCSD_FP64 && !(c->precision == CCSD_MIXED && c->polish_precision == CCSD_OZAKI))
        return refuse("polish_precision must be CCSD_FP64, or CCSD_OZAKI for a CCSD_MIXED config");
    if (c->precision == CCSD_OZAKI || c->polish_precision == CCSD_OZAKI) {
        if (c->oz_slices != 0 && (c->oz_slices < 3 || c->oz_slices > OZ_MAX_SLICES))
            return refuse("oz_slices must be 0 or 3..8");
        if (c->nvir > 96) return refuse("the Ozaki form needs nvir <= 96");   // one W' row (v^2 complex) in shared memory
    }
    if (c->diis_depth < 0 || c->diis_depth == 1 || c->diis_depth > 8) return refuse("diis_depth must be 0 or 2..8");
    if (c->max_iter < 0) return refuse("max_iter must be >= 0");
    if (!(c->conv_tol >= 0.0) || !std::isfinite(c->conv_tol)) return refuse("conv_tol must be finite and >= 0");
    if (c->precision == CCSD_MIXED && (!(c->mixed_tol >= 0.0) || !std::isfinite(c->mixed_tol)))
        return refuse("mixed_tol must be finite and >= 0");
    if (c->lean != 0 && c->lean != 1) return refuse("lean must be 0 or 1");
    const long long N = (long long)c->nk_dims[0] * c->nk_dims[1] * c->nk_dims[2];
    const long long vvvv = (long long)c->nvir * c->nvir * c->nvir * c->nvir;
    if (vvvv * 1 > (1LL << 30)) return refuse("nvir^4 must be <= 2^30 (32-bit offsets inside a block)");
    if (N * N * N * vvvv > (1LL << 40)) return refuse("N_k^3 nvir^4 must be <= 2^40");
    return true;
}

// Host ranges this library registered as mapped pinned memory (host vvvv read in
// place), counted per handle: several live handles may share one host array, and
// the range is unregistered when the last of them is destroyed.  A range the caller
// registered is never unregistered here.
struct HostReg { size_t bytes; int handles; };
std::mutex g_host_reg_mu;
std::map<void*, HostReg> g_host_reg;

// 1: registered (or counted) by the library; 0: already registered by the caller;
// < 0: error code.
int host_register(void* p, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_host_reg_mu);
    auto it = g_host_reg.find(p);
    if (it != g_host_reg.end()) {
        if (bytes > it->second.bytes) return CCSD_ERR_INVALID;   // a longer range from the same start
        ++it->second.handles;
        return 1;
    }
    const cudaError_t e = cudaHostRegister(p, bytes, cudaHostRegisterMapped);
    if (e == cudaSuccess) { g_host_reg[p] = HostReg{bytes, 1}; return 1; }
    cudaGetLastError();
    return e == cudaErrorHostMemoryAlreadyRegistered ? 0 : CCSD_ERR_CUDA;
}

void host_unregister(void* p) {
    std::lock_guard<std::mutex> lock(g_host_reg_mu);
    auto it = g_host_reg.find(p);
    if (it == g_host_reg.end()) return;
    if (--it->second.handles == 0) {
        cudaHostUnregister(p);
        g_host_reg.erase(it);
    }
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Fills a handle whose cfg, grid and sizes are set: inputs (device ones borrowed, host
// ones copied), amplitudes, work buffers, DIIS history, Fock diagonals, the residual
// plan and its tables.  With al.dry nothing is allocated, copied or launched and
// h->owned_bytes ends as the device memory ccsd_create would take (ins may be null).
int setup_handle(ccsd_ctx* h, Alloc& al, const void* const* ins, const bool* on_dev, int int_dtype,
                 bool vvvv_on_host) {
    const long long N = h->N, o = h->o, v = h->v, N3 = N * N * N;
    const long long sizes[9] = {N * o * o, N * v * v, N * o * v, N3 * o * o * o * o, N3 * o * o * o * v,
                                N3 * o * o * v * v, N3 * o * o * v * v, N3 * o * v * v * v, N3 * v * v * v * v};
    for (int i = 0; i < 9; ++i) {
        const bool c64 = i >= 3 && int_dtype == CCSD_C64;
        const size_t bytes = (size_t)sizes[i] * (c64 ? 8 : 16);
        void* d = nullptr;
        if (on_dev[i]) {
            d = al.dry ? (void*)(uintptr_t)256 : const_cast<void*>(ins[i]);
        } else if (i == 8 && vvvv_on_host) {
            // vvvv read in place from host memory (mapped, pinned): no device copy
            if (al.dry) {
                d = (void*)(uintptr_t)256;
            } else {
                void* hp = const_cast<void*>(ins[i]);
                const int r = host_register(hp, bytes);
                if (r < 0) return r;
                if (r == 1) h->host_registered = hp;
                if (cudaHostGetDevicePointer(&d, hp, 0) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_CUDA; }
            }
        } else {
            d = al.get(bytes);
            if (!d) return al.err;
            if (!al.dry && cudaMemcpyAsync(d, ins[i], bytes, cudaMemcpyHostToDevice, h->st) != cudaSuccess) return CCSD_ERR_CUDA;
        }
        if (c64) { h->shadow[B_FOO_IN + i] = (float2*)d; h->in32[B_FOO_IN + i] = true; }
        else h->buf[B_FOO_IN + i] = (double2*)d;
    }
    auto dalloc = [&](long long n) { return (double2*)al.get((size_t)n * 16); };
    h->amp = dalloc(h->n1 + h->n2);
    h->res = dalloc(h->n1 + h->n2);
    if (!h->amp || !h->res) return al.err;
    h->buf[B_T1] = h->amp; h->buf[B_T2] = h->amp + h->n1;
    h->buf[B_R1] = h->res; h->buf[B_R2] = h->res + h->n1;
    h->buf[B_TAU] = dalloc(h->n2); h->buf[B_TAUT] = dalloc(h->n2);
    h->buf[B_FOV] = dalloc(N * o * v); h->buf[B_FOO] = dalloc(N * o * o); h->buf[B_FVV] = dalloc(N * v * v);
    h->buf[B_FOOP] = dalloc(N * o * o); h->buf[B_FVVP] = dalloc(N * v * v);
    h->buf[B_WHH] = dalloc(N3 * o * o * o * o);
    h->buf[B_WRING] = dalloc(h->n2);
    h->buf[B_Q] = dalloc(N3 * o * o * o * v);
    h->buf[B_TT] = dalloc(N3 * o * o * o * v);
    h->buf[B_ZR] = dalloc(h->n2);
    if (al.err) return al.err;
    if (h->cfg.diis_depth > 0) {
        // canonical blocks of the DIIS history (t2 antisymmetry, paper Sec. 2)
        std::vector<int> cblk, cmap;
        std::vector<double> cw;
        if (!diis_canonical_blocks(h->kg, cblk, cw, cmap)) return CCSD_ERR_INVALID;
        h->nc = (long long)cblk.size();
        std::vector<int> ctgt;                 // the full blocks each canonical block is written to
        if (!diis_canonical_targets(cmap, h->nc, ctgt)) return CCSD_ERR_INVALID;
        h->d_cblk = upload(al, cblk, h->st);
        h->d_cw = upload(al, cw, h->st);
        h->d_ctgt = upload(al, ctgt, h->st);
        const long long np = h->n1 + h->nc * o * o * v * v;
        for (int d = 0; d < h->cfg.diis_depth; ++d) {
            h->hx.push_back(dalloc(np));
            h->he.push_back(dalloc(np));
        }
        h->d_diis = (DiisState*)al.get(sizeof(DiisState));
        h->d_diis_part = (double*)al.get(sizeof(double) * (size_t)h->cfg.diis_depth * kRedBlocks);
        if (al.err) return al.err;
        memset(&h->diis_init, 0, sizeof h->diis_init);
        h->diis_init.depth = h->cfg.diis_depth;
        for (int d = 0; d < h->cfg.diis_depth; ++d) { h->diis_init.hx[d] = h->hx[(size_t)d]; h->diis_init.he[d] = h->he[(size_t)d]; }
        if (!al.dry && cudaMemcpyAsync(h->d_diis, &h->diis_init, sizeof(DiisState), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return CCSD_ERR_CUDA;
    }
    if (al.err) return al.err;
    if (!al.dry && cudaMemsetAsync(h->amp, 0, (size_t)(h->n1 + h->n2) * 16, h->st) != cudaSuccess) return CCSD_ERR_CUDA;

    // Fock diagonals and the fourth momentum of doubles blocks
    {
        std::vector<double> eo((size_t)(N * o)), ev((size_t)(N * v));
        if (!al.dry) {
            std::vector<double2> foo((size_t)(N * o * o)), fvv((size_t)(N * v * v));
            if (cudaMemcpyAsync(foo.data(), h->buf[B_FOO_IN], foo.size() * 16, cudaMemcpyDefault, h->st) != cudaSuccess ||
                cudaMemcpyAsync(fvv.data(), h->buf[B_FVV_IN], fvv.size() * 16, cudaMemcpyDefault, h->st) != cudaSuccess ||
                cudaStreamSynchronize(h->st) != cudaSuccess) return CCSD_ERR_CUDA;
            for (long long k = 0; k < N; ++k) {
                for (long long i = 0; i < o; ++i) eo[(size_t)(k * o + i)] = foo[(size_t)((k * o + i) * o + i)].x;
                for (long long a = 0; a < v; ++a) ev[(size_t)(k * v + a)] = fvv[(size_t)((k * v + a) * v + a)].x;
            }
            for (double x : eo) for (double y : ev) if (!(x - y < 0.0 || x - y > 0.0)) return CCSD_ERR_INVALID;
        }
        h->eo = upload(al, eo, h->st);
        h->ev = upload(al, ev, h->st);
        std::vector<int> kb((size_t)N3);
        for (int ki = 0; ki < N; ++ki) for (int kj = 0; kj < N; ++kj) for (int ka = 0; ka < N; ++ka)
            kb[(size_t)(((long long)ki * N + kj) * N + ka)] = h->kg.k4(ki, kj, ka);
        h->kb_of = upload(al, kb, h->st);
        if (al.err) return al.err;
        if (h->cfg.diis_depth > 0) {
            const long long np = h->n1 + h->nc * (long long)o * o * v * v;
            h->d_rden = (double*)al.get((size_t)np * sizeof(double));
            if (al.err) return al.err;
            if (!al.dry)
                op_kernel<DiisRdenOp><<<ew_grid(np), 256, 0, h->st>>>(DiisRdenOp{h->d_rden, h->d_cblk, h->nc, h->eo,
                                                                                  h->ev, h->kb_of, (int)N, (int)o,
                                                                                  (int)v});
        }
    }
    set_sizes(h);
    size_t work_need = 0;
    int rc = build_plan(h, al, work_need);
    if (rc) return rc;
    if (h->cfg.precision == CCSD_MIXED) {
        // GEMM steps that a mixed handle runs in FP32 (all but the FP64-only ones)
        for (const Step& st : h->seq) {
            if (st.kind != 0 || st.mode == 1 || st.mode == 4) continue;
            const GemmArgs& g32 = h->gemms[st.idx].args32;
            if (g32.nsplit > 1) work_need = std::max(work_need, (size_t)g32.nsplit * g32.nbatch * g32.M * g32.N);
        }
    }
    if (work_need) { h->work = dalloc((long long)work_need); if (!h->work) return al.err; }
    if (h->oz_work_elems) { h->oz_work = dalloc(h->oz_work_elems); if (!h->oz_work) return al.err; }
    h->work_elems = work_need;
    h->red_blocks = kRedBlocks;
    h->red = (double*)al.get(sizeof(double) * h->red_blocks);
    h->red_out = (double*)al.get(sizeof(double) * 4);
    h->cred = (double2*)al.get(sizeof(double2) * h->red_blocks);
    h->cred_out = (double2*)al.get(sizeof(double2) * 2);
    return al.err;
}

void init_ctx(ccsd_ctx* h, const ccsd_config* cfg) {
    h->cfg = *cfg;
    h->kg.init(cfg->nk_dims);
    h->N = h->kg.N; h->o = cfg->nocc; h->v = cfg->nvir;
    if (cfg->lean) {    // W' slabs of about a third of the momentum pairs
        const long long N = h->N, v = h->v;
        h->wab_cap_bytes = 16 * N * v * v * v * v * std::max<long long>(1, (N * (N + 1) / 2 + 2) / 3);
    }
    h->fp32 = cfg->precision == CCSD_MIXED ? 1 : 0;
    h->oz_on = cfg->precision == CCSD_OZAKI ? 1 : 0;
    h->has_oz = cfg->precision == CCSD_OZAKI || (cfg->precision == CCSD_MIXED && cfg->polish_precision == CCSD_OZAKI);
    h->oz_slices = cfg->oz_slices ? cfg->oz_slices : 7;
    const long long N = h->N;
    h->n1 = N * h->o * h->v;
    h->n2 = N * N * N * h->o * h->o * h->v * h->v;
}

// Device bytes ccsd_create takes for this config, from a dry run of its setup; 0 on error.
size_t footprint_bytes(const ccsd_config* c, const bool* on_dev, int int_dtype, bool vvvv_on_host = false) {
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return 0;
    init_ctx(h, c);
    Alloc al{h};
    al.dry = true;
    const int rc = setup_handle(h, al, nullptr, on_dev, int_dtype, vvvv_on_host);
    const size_t b = rc ? 0 : h->owned_bytes;
    delete h;
    return b;
}

}  // namespace

// First half of an iteration: residual and max|R| on the device, the norm
// copied into pinned host memory; returns without waiting.
int iter_begin(ccsd_ctx* h) {
    int rc = run_residual_async(h);
    if (rc) return rc;
    const long long n = h->n1 + h->n2;
    maxabs_partial<<<h->red_blocks, 256, 0, h->st>>>(MaxabsOp{h->res, n, h->red});
    final_max<<<1, 32, 0, h->st>>>(h->red, h->red_blocks, h->red_out);
    h->launches += 2;
    CK(cudaMemcpyAsync(h->norm_host, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaEventRecord(h->ev_norm, h->st));
    return 0;
}

// Second half: waits for the norm, then the convergence test and the update
// t <- t + R/D (plus DIIS) unless converged.
int iter_finish(ccsd_ctx* h, double mr, int* done);

// The convergence test alone: CCSD_ERR_DIVERGED for a non-finite max|R|, *done when
// max|R| < conv_tol.
int iter_test(const ccsd_ctx* h, double mr, int* done) {
    *done = 0;
    if (!std::isfinite(mr)) { refuse("max|R| is not finite: the iteration diverged"); return CCSD_ERR_DIVERGED; }
    if (mr < h->cfg.conv_tol) *done = 1;
    return CCSD_OK;
}

int iter_end(ccsd_ctx* h, int* done, double* max_resid) {
    *done = 0;
    CK(cudaEventSynchronize(h->ev_norm));
    int rc = check_tc_err(h);
    if (rc) return rc;
    if (h->trace && (rc = trace_collect(h, 0, h->seq.size()))) return rc;
    const double mr = *h->norm_host;
    *max_resid = mr;
    return iter_finish(h, mr, done);
}

// The convergence test on max|R| = mr and, unless converged, the update t <- t + R/D
// with DIIS extrapolation (enqueued on the handle's stream; the DIIS inner products
// synchronize it).
int iter_finish(ccsd_ctx* h, double mr, int* done) {
    int rc = iter_test(h, mr, done);
    if (rc || *done) return rc;
    const long long n = h->n1 + h->n2;
    const int depth = h->cfg.diis_depth;
    const size_t tu = h->seq.size();     // trace slot of the update
    if (h->trace) cudaEventRecord(h->ev0[tu], h->st);
    if (depth == 0) {
        update_kernel<<<ew_grid(n), 256, 0, h->st>>>(update_op(h, nullptr));
        ++h->launches;
        if (h->trace) { cudaEventRecord(h->ev1[tu], h->st); if ((rc = trace_collect(h, tu, tu + 1))) return rc; }
    } else {
        // DIIS on the device: pack x = t + R/D and e = R/D into the history, inner products
        // of e with the filled slots, the Pulay solve, the extrapolation (no host round trip)
        const long long blk = (long long)h->o * h->o * h->v * h->v;
        const long long np = h->n1 + h->nc * blk;
        op_kernel<DiisPackOp><<<ew_grid(np), 256, 0, h->st>>>(DiisPackOp{h->amp, h->res, h->d_diis, h->d_cblk, h->nc,
                                                                          h->d_rden, h->N, h->o, h->v, nullptr});
        op_kernel<DiisDotOp><<<(unsigned)h->red_blocks, 256, 0, h->st>>>(
            DiisDotOp{h->d_diis, h->n1, blk, h->nc, h->d_cw, h->d_diis_part, h->red_blocks, nullptr});
        op_kernel<DiisSolveOp><<<1, 32, 0, h->st>>>(DiisSolveOp{h->d_diis, h->d_diis_part, h->red_blocks, nullptr});
        const DiisComboOp cb{h->amp, h->d_diis, h->d_ctgt, h->nc, h->N, h->o, h->v, nullptr};
        op_kernel<DiisComboOp><<<(unsigned)std::min<long long>(cb.units(), 8LL * kSMs), 256, 0, h->st>>>(cb);
        h->launches += 4;
        if (h->trace) { cudaEventRecord(h->ev1[tu], h->st); if ((rc = trace_collect(h, tu, tu + 1))) return rc; }
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { last_err(ce); return CCSD_ERR_CUDA; }
    return CCSD_OK;
}


// ================================================================ serving form
// A host thread admits submitted solves by device-memory footprint (each gets a
// handle whose integrals and amplitudes stay resident until it finishes) and
// advances all admitted solves in rounds.  A round is one iteration of every
// admitted solve: the solves are partitioned into groups of equal plan signature,
// precision state and contraction tile shapes, every step of the residual is ONE
// grouped launch per group (the groups on streams of their own, forked from the
// server's stream), all max|R| come back in one copy, and then each solve takes its
// convergence test and update (with DIIS).  Group members keep the split-K choices
// of their own plans, so a solve's iterates are bitwise those it has alone.  Solves
// in the Ozaki arithmetic run their residual on their own.  Converged solves retire,
// free their memory and make room for the queue; a group is rebuilt only when its
// membership changes.
namespace {

struct ServerReq {
    uint64_t id = 0;
    ccsd_config cfg{};
    ccsd_inputs in{};
    int state = 0;                 // 0 queued, 1 running, 2 done, < 0 error code
    int phase = 0;                 // mixed form: 0 mixed iterations, 1 FP64 polish
    int iters = 0, polish_left = 0;
    double e_re = 0.0, e_im = 0.0, max_resid = 0.0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    size_t bytes = 0;
    int lane = 0;                  // cost class of one iteration (its lane of rounds)
    ccsd_t h = nullptr;
};

// A lane runs rounds over the solves of one cost class, on a stream of its own, at its
// own pace: a round of small solves does not wait for the iteration of a large one.
struct Lane {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;    // recorded after the round's norms are copied out
    cudaEvent_t fork = nullptr;
    std::vector<cudaStream_t> gst; // one stream per group of the round
    std::vector<cudaEvent_t> gev;
    std::vector<ServerReq*> active;
    std::vector<ServerReq*> incoming;  // admitted while a round was in flight: join the next one
    std::map<std::vector<long long>, std::unique_ptr<Group>> groups;
    // the round in flight
    bool in_flight = false;
    std::vector<std::pair<Group*, std::vector<ServerReq*>>> grp;
    std::vector<int> first;
    std::vector<ServerReq*> solo;
    std::vector<int> began;
    double* h_norms = nullptr;     // pinned, one per slot
    double t0 = 0.0, t_built = 0.0;
    long long builds = 0;
};

constexpr int kLanes = 4;

}  // namespace

struct ccsd_server {
    size_t budget = 0, used = 0;
    int max_slots = 1;
    int device = 0;
    cudaStream_t st = nullptr;     // every device operation of the server
    bool own_stream = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServerReq*> pending;
    std::vector<ServerReq*> active;
    std::map<uint64_t, ServerReq*> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
    std::chrono::steady_clock::time_point t0;
    // lanes of grouped rounds (touched by the loop thread only)
    Lane lanes[kLanes];
    cudaEvent_t start = nullptr;   // the lanes' streams wait on it: work queued on st before
    ChunkPool pool;                // device chunks of the groups' tables
    long long rounds = 0, grouped_launches = 0, rebuilds = 0, finished = 0;
    double round_s = 0.0, rebuild_s = 0.0, wait_s = 0.0, run_s = 0.0;
};

namespace {

double server_now(const ccsd_server* S) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

size_t request_bytes(const ccsd_config& c, const ccsd_inputs& in) {
    const void* ins[9] = {in.f_oo, in.f_vv, in.f_ov, in.oooo, in.ooov, in.oovv, in.ovvo, in.ovvv, in.vvvv};
    bool on_dev[9];
    for (int i = 0; i < 9; ++i) on_dev[i] = is_device_ptr(ins[i]);
    return footprint_bytes(&c, on_dev, in.int_dtype, in.vvvv_on_host != 0);
}

// Fields that ccsd_poll reads (state, energy, iterations, max|R|) change only under S->mu.
void server_finish(ccsd_server* S, ServerReq* r, int state) {
    double e_re = 0.0, e_im = 0.0;
    if (r->h) {
        if (state == 2) {
            // a failed energy reduction ends the request with its code, not as converged
            const int rc = ccsd_energy(r->h, &e_re, &e_im);
            if (rc) { state = rc; e_re = e_im = 0.0; }
        }
        ccsd_destroy(r->h);
        r->h = nullptr;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    r->e_re = e_re;
    r->e_im = e_im;
    r->t_done = server_now(S);
    r->state = state;
    S->used -= r->bytes;
    if (r->t_admit > 0.0) {
        S->finished += 1;
        S->wait_s += r->t_admit - r->t_submit;
        S->run_s += r->t_done - r->t_admit;
    }
}

// Grouping key of a solve in its current arithmetic: solves with equal keys share every
// grouped launch of a round.
std::vector<long long> server_key(const ccsd_ctx* h) {
    std::vector<long long> k{h->fp32, h->oz_on, h->cfg.precision};
    for (const Step& st : h->seq) {
        k.push_back(st.kind * 16 + st.mode);
        if (st.kind == 0) k.push_back(h->gemms[st.idx].cfg);
    }
    return k;
}

// Builds the groups of a lane's round (reusing those whose membership is unchanged);
// Ozaki-arithmetic solves go to `solo`.
int lane_groups(ccsd_server* S, Lane& L, std::vector<std::pair<Group*, std::vector<ServerReq*>>>& out,
                std::vector<ServerReq*>& solo, long long* builds) {
    std::map<std::vector<long long>, std::vector<ServerReq*>> parts;
    for (ServerReq* r : L.active) {
        if (r->h->oz_on) solo.push_back(r);
        else parts[server_key(r->h)].push_back(r);
    }
    std::map<std::vector<long long>, std::unique_ptr<Group>> next;
    int rc = 0;
    for (auto& kv : parts) {
        std::vector<ccsd_ctx*> hs;
        std::vector<uint64_t> ids;
        for (ServerReq* r : kv.second) { hs.push_back(r->h); ids.push_back(r->id); }
        // a group is reused only for exactly the same requests: its device tables hold
        // their buffers' addresses
        auto it = L.groups.find(kv.first);
        if (it != L.groups.end() && it->second->rids == ids && it->second->m == hs) {
            next[kv.first] = std::move(it->second);
        } else {
            std::unique_ptr<Group> G(new (std::nothrow) Group());
            if (!G) return CCSD_ERR_OOM;
            G->pool = &S->pool;
            G->m = hs;
            G->rids = ids;
            ++*builds;
            if ((rc = group_alloc(*G, sizeof(int) * hs.size(), (void**)&G->d_skip)) ||
                (rc = group_build(*G, hs[0]->fp32, {}, nullptr, G->d_skip, L.st, true))) {
                group_free(*G);
                return rc;
            }
            next[kv.first] = std::move(G);
        }
        out.emplace_back(next[kv.first].get(), kv.second);
    }
    for (auto& kv : L.groups) if (kv.second) group_free(*kv.second);
    L.groups = std::move(next);
    while (L.gst.size() < out.size()) {
        cudaStream_t gs = nullptr;
        cudaEvent_t ge = nullptr;
        if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_CUDA; }
        L.gst.push_back(gs);
        if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return CCSD_ERR_CUDA; }
        L.gev.push_back(ge);
    }
    return 0;
}

// Completes one solve's iteration from its max|R| (convergence test, update, phase
// changes); false if the request finished.
bool server_complete(ccsd_server* S, ServerReq* r, int rc, int done, double mr) {
    int iters = 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        r->max_resid = mr;
        if (!rc && !done) iters = ++r->iters;
    }
    if (rc) { server_finish(S, r, rc); return false; }
    if (!done) {
        if (iters >= r->cfg.max_iter) { server_finish(S, r, CCSD_ERR_NOT_CONVERGED); return false; }
        if (r->phase == 1 && --r->polish_left <= 0) { server_finish(S, r, 2); return false; }
        return true;
    }
    if (r->phase == 0 && r->polish_left > 0) {    // mixed phase done: FP64 (or Ozaki) polish
        r->phase = 1;
        const int prc = ccsd_set_precision(r->h, r->cfg.polish_precision == CCSD_OZAKI ? CCSD_OZAKI : CCSD_FP64);
        if (prc) { server_finish(S, r, prc); return false; }
        r->h->cfg.conv_tol = r->cfg.conv_tol;
        return true;
    }
    server_finish(S, r, 2);
    return false;
}

// Lane of a solve: the order of magnitude of its iteration's flops (four classes).
int lane_of(const ccsd_config& c) {
    const double N = (double)c.nk_dims[0] * c.nk_dims[1] * c.nk_dims[2], o = c.nocc, v = c.nvir;
    const double fl = 8.0 * N * N * N * N * (o * o * v * v * v * v + 2 * o * o * o * v * v * v + 2 * o * o * o * o * v * v);
    const int l = (int)std::floor(std::log10(std::max(fl, 1.0))) - 9;
    return std::max(0, std::min(kLanes - 1, l));
}

// Launches one round of lane L (residuals and norms of every solve; no host wait).
void lane_launch(ccsd_server* S, Lane& L) {
    L.grp.clear();
    L.solo.clear();
    L.first.clear();
    L.builds = 0;
    L.t0 = server_now(S);
    int grc = lane_groups(S, L, L.grp, L.solo, &L.builds);
    L.t_built = server_now(S) - L.t0;
    if (grc) {                                 // groups could not be built: fail the lane's solves
        for (ServerReq* r : L.active) server_finish(S, r, grc);
        L.active.clear();
        L.grp.clear();
        L.solo.clear();
        return;
    }
    cudaEventRecord(L.fork, L.st);
    int slot = 0;
    for (size_t g = 0; g < L.grp.size(); ++g) {
        Group& G = *L.grp[g].first;
        cudaStreamWaitEvent(L.gst[g], L.fork, 0);
        group_residual(G, L.gst[g]);
        G.norms.fn(L.gst[g]);
        L.first.push_back(slot);
        cudaMemcpyAsync(L.h_norms + slot, G.d_norms, sizeof(double) * G.m.size(), cudaMemcpyDeviceToHost, L.gst[g]);
        slot += (int)G.m.size();
        cudaEventRecord(L.gev[g], L.gst[g]);
        cudaStreamWaitEvent(L.st, L.gev[g], 0);
        S->grouped_launches += group_launches(G, false);
    }
    L.began.assign(L.solo.size(), 0);
    for (size_t i = 0; i < L.solo.size(); ++i) L.began[i] = iter_begin(L.solo[i]->h);
    cudaEventRecord(L.done, L.st);
    L.in_flight = true;
}

// Completes lane L's round once its norms have arrived: each solve's convergence test,
// one grouped update of the solves that go on, retirements.
void lane_complete(ccsd_server* S, Lane& L) {
    L.in_flight = false;
    int src = cudaEventSynchronize(L.done) == cudaSuccess ? 0 : CCSD_ERR_CUDA;
    if (src) last_err(cudaGetLastError());
    std::vector<ServerReq*> keep;
    for (size_t g = 0; g < L.grp.size(); ++g) {
        Group& G = *L.grp[g].first;
        const int rc = src ? src : group_check_err(G, L.st);
        const size_t nm = L.grp[g].second.size();
        std::vector<int> frc(nm, 0), done(nm, 0), skip(nm, 1);
        for (size_t i = 0; i < nm; ++i) {
            const double mr = L.h_norms[L.first[g] + i];
            frc[i] = rc ? rc : iter_test(L.grp[g].second[i]->h, mr, &done[i]);
            skip[i] = (frc[i] || done[i]) ? 1 : 0;
        }
        int urc = rc;
        if (!urc && cudaMemcpyAsync(G.d_skip, skip.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, L.st) != cudaSuccess) {
            last_err(cudaGetLastError());
            urc = CCSD_ERR_CUDA;
        }
        if (!urc) {
            G.update.fn(L.st);
            if (cudaGetLastError() != cudaSuccess) urc = CCSD_ERR_CUDA;
        }
        for (size_t i = 0; i < nm; ++i) {
            ServerReq* r = L.grp[g].second[i];
            const int code = frc[i] ? frc[i] : (urc && !done[i]) ? urc : 0;
            if (server_complete(S, r, code, done[i], L.h_norms[L.first[g] + i])) keep.push_back(r);
        }
    }
    for (size_t i = 0; i < L.solo.size(); ++i) {
        ServerReq* r = L.solo[i];
        int done = 0, rc = L.began[i];
        double mr = 0.0;
        if (!rc) rc = iter_end(r->h, &done, &mr);
        if (server_complete(S, r, rc, done, mr)) keep.push_back(r);
    }
    keep.insert(keep.end(), L.incoming.begin(), L.incoming.end());
    L.incoming.clear();
    L.active = keep;
    L.grp.clear();
    L.solo.clear();
    std::lock_guard<std::mutex> lock(S->mu);
    S->rounds += 1;
    S->rebuilds += L.builds;
    S->rebuild_s += L.t_built;
    S->round_s += server_now(S) - L.t0;
}

void server_loop(ccsd_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<ServerReq*> admit;
        bool busy = false;
        for (const Lane& L : S->lanes) busy = busy || !L.active.empty() || !L.incoming.empty() || L.in_flight;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            if (!busy) S->cv.wait(lock, [&] { return S->stop || !S->pending.empty(); });
            if (S->stop && !busy && S->pending.empty()) break;
            if (S->stop) {                         // cancel what has not started
                for (ServerReq* r : S->pending) { r->state = CCSD_ERR_INVALID; r->t_done = server_now(S); }
                S->pending.clear();
            }
            while (!S->pending.empty() && (int)(S->active.size() + admit.size()) < S->max_slots) {
                ServerReq* r = S->pending.front();
                if (r->bytes > S->budget) {        // can never fit
                    S->pending.pop_front();
                    r->state = CCSD_ERR_OOM;
                    r->t_done = server_now(S);
                    continue;
                }
                if (S->used + r->bytes > S->budget) break;     // FIFO: wait for memory
                S->pending.pop_front();
                S->used += r->bytes;
                admit.push_back(r);
            }
        }
        for (ServerReq* r : admit) {
            r->lane = lane_of(r->cfg);
            int rc = ccsd_create(&r->cfg, &r->in, S->lanes[r->lane].st, &r->h);
            if (rc) { server_finish(S, r, rc); continue; }
            r->polish_left = r->cfg.precision == CCSD_MIXED ? r->cfg.polish_iters : 0;
            if (r->cfg.precision == CCSD_MIXED) r->h->cfg.conv_tol = std::max(r->cfg.mixed_tol, r->cfg.conv_tol);
            Lane& L = S->lanes[r->lane];
            (L.in_flight ? L.incoming : L.active).push_back(r);
            std::lock_guard<std::mutex> lock(S->mu);
            r->t_admit = server_now(S);
            r->state = 1;
            S->active.push_back(r);
        }
        // every lane at its own pace: complete the rounds whose norms have arrived, start
        // the next round of every idle lane with solves
        bool progressed = !admit.empty();
        for (Lane& L : S->lanes) {
            if (L.in_flight) {
                const cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) cudaGetLastError();
                lane_complete(S, L);
                progressed = true;
            }
            if (!L.in_flight && !L.active.empty()) { lane_launch(S, L); progressed = true; }
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            std::vector<ServerReq*> act;
            for (const Lane& L : S->lanes) {
                act.insert(act.end(), L.active.begin(), L.active.end());
                act.insert(act.end(), L.incoming.begin(), L.incoming.end());
            }
            S->active = act;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (Lane& L : S->lanes) {
        for (auto& kv : L.groups) if (kv.second) group_free(*kv.second);
        L.groups.clear();
    }
}

}  // namespace

extern "C" {

int ccsd_footprint(const ccsd_config* cfg, int inputs_on_device, int int_dtype, size_t* bytes) {
    ApiScope api_scope_;
    if (!valid_cfg(cfg) || !bytes || (int_dtype != CCSD_C128 && int_dtype != CCSD_C64)) return CCSD_ERR_INVALID;
    bool on_dev[9];
    for (bool& x : on_dev) x = inputs_on_device != 0;
    *bytes = footprint_bytes(cfg, on_dev, int_dtype);
    return *bytes ? CCSD_OK : CCSD_ERR_INVALID;
}


int ccsd_plan_describe(const ccsd_config* cfg, int max_steps, int* kinds, int* modes, double* flops,
                       const char** names, int* n_steps) {
    ApiScope api_scope_;
    if (!valid_cfg(cfg) || max_steps < 0 || !n_steps) return CCSD_ERR_INVALID;
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return CCSD_ERR_OOM;
    init_ctx(h, cfg);
    set_sizes(h);
    Alloc al{h};
    al.dry = true;
    size_t work_need = 0;
    const int rc = build_plan(h, al, work_need);
    *n_steps = (int)h->seq.size();
    for (int i = 0; i < (int)h->seq.size() && i < max_steps; ++i) {
        if (kinds) kinds[i] = h->seq[i].kind;
        if (modes) modes[i] = h->seq[i].mode;
        if (flops) flops[i] = h->seq[i].flops;
        if (names) names[i] = h->seq[i].name;    // static strings
    }
    delete h;
    return rc;
}

int ccsd_plan_check(const ccsd_config* cfg, long long* n_launches, size_t* table_bytes) {
    ApiScope api_scope_;
    if (!valid_cfg(cfg)) return CCSD_ERR_INVALID;
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return CCSD_ERR_OOM;
    init_ctx(h, cfg);
    set_sizes(h);
    Alloc al{h};
    al.dry = true;
    size_t work_need = 0;
    const int rc = build_plan(h, al, work_need);
    long long n = 0;
    for (const Step& st : h->seq)
        n += ((st.kind == 0 && h->gemms[st.idx].args.nsplit > 1) || (st.kind == 6 && h->tcs[st.idx].oz &&
              h->tcs[st.idx].z.nsplit > 1)) ? 2 : 1;
    if (n_launches) *n_launches = n;
    if (table_bytes) *table_bytes = h->owned_bytes;
    delete h;
    return rc;
}

}  // extern "C"

namespace {

// The tensor-core self-test; skip_stage >= 0 leaves that pipeline stage unloaded
// (with a short wait limit) to exercise the bounded-wait failure path.
int tc_selftest_impl(int M, int Ncols, int K, int nterms, unsigned long long seed, int skip_stage, double* rel_err) {
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return CCSD_ERR_OOM;
    h->cfg.precision = CCSD_MIXED;
    Alloc al{h};
    auto fail = [&](int code) { ccsd_destroy(h); return code; };
    const long long nA = (long long)M * K, nB = (long long)Ncols * K, nC = (long long)M * Ncols;
    // random complex operands on the host, uniform in [-1, 1)
    std::vector<double2> hA((size_t)nA), hB((size_t)nB);
    unsigned long long x = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto rnd = [&]() { x = x * 6364136223846793005ULL + 1442695040888963407ULL; return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0; };
    for (auto& z : hA) { z.x = rnd(); z.y = rnd(); }
    for (auto& z : hB) { z.x = rnd(); z.y = rnd(); }
    h->buf[B_STA] = upload(al, hA, h->st); h->bufsize[B_STA] = nA;
    h->buf[B_STB] = upload(al, hB, h->st); h->bufsize[B_STB] = nB;
    h->buf[B_ZR] = (double2*)al.get((size_t)nC * 16); h->bufsize[B_ZR] = nC;
    h->buf[B_TAU] = (double2*)al.get((size_t)nC * 16); h->bufsize[B_TAU] = nC;
    h->tc_err = (int*)al.get(sizeof(int));
    if (al.err) return fail(al.err);
    if (cudaMemsetAsync(h->buf[B_ZR], 0, (size_t)nC * 16, h->st) != cudaSuccess ||
        cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    // reference: FP64 SIMT engine, C_ref = A B^T
    size_t work_need = 0;
    GemmSpec g; g.a = B_STA; g.b = B_STB; g.c = B_TAU; g.acc = false;
    g.M = M; g.N = Ncols; g.K = K; g.nbatch = 1; g.nchunk = 1;
    g.offA = {0}; g.offB = {0}; g.offC = {0};
    g.rowA = tab({{M, K}}); g.colA = tab({{K, 1}});
    g.rowB = tab({{K, 1}}); g.colB = tab({{Ncols, K}});
    g.rowC = tab({{M, Ncols}}); g.colC = tab({{Ncols, 1}});
    int rc = finalize_gemm(h, al, g, work_need);
    if (rc) return fail(rc);
    if (work_need) { h->work = (double2*)al.get(work_need * 16); if (!h->work) return fail(al.err); }
    // tensor cores: embed, GEMM
    const int kpad = (2 * K + TC_BK - 1) / TC_BK * TC_BK;
    TcBuf ta{}, tb{};
    if ((rc = tc_alloc(h, al, ta, M, kpad)) || (rc = tc_alloc(h, al, tb, 2LL * Ncols, kpad))) return fail(rc);
    if ((rc = add_embed(h, al, B_STA, ta, 0, M, K, {0}, tab({{M, K}}), tab({{K, 1}}), false)) ||
        (rc = add_embed(h, al, B_STB, tb, 1, Ncols, K, {0}, tab({{Ncols, K}}), tab({{K, 1}}), false)))
        return fail(rc);
    std::vector<long long> oc;
    for (int m = 0; m < M; ++m) oc.push_back((long long)m * Ncols);
    if ((rc = add_tc(h, al, ta, tb, B_ZR, M, 2 * Ncols, 1, 1, {0}, {0}, oc, tab({{Ncols, 1}}), 1.0, nterms)))
        return fail(rc);
    if (skip_stage >= 0) {
        h->tcs[0].a.skip_stage = skip_stage;
        h->tcs[0].a.spin_limit = 1LL << 14;
    }
    launch_gemm(h, h->gemms[0]);
    launch_embed(h, h->embeds[0]);
    launch_embed(h, h->embeds[1]);
    launch_tc(h, h->tcs[0]);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    int flag = 0;
    std::vector<double2> c1((size_t)nC), c2((size_t)nC);
    if (cudaMemcpy(&flag, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(c1.data(), h->buf[B_ZR], (size_t)nC * 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(c2.data(), h->buf[B_TAU], (size_t)nC * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CCSD_ERR_CUDA);
    if (flag) return fail(CCSD_ERR_TIMEOUT);
    double num = 0.0, den = 0.0;
    for (long long i = 0; i < nC; ++i) {
        num = std::max(num, std::hypot(c1[(size_t)i].x - c2[(size_t)i].x, c1[(size_t)i].y - c2[(size_t)i].y));
        den = std::max(den, std::hypot(c2[(size_t)i].x, c2[(size_t)i].y));
    }
    *rel_err = den > 0 ? num / den : num;
    ccsd_destroy(h);
    return CCSD_OK;
}

// C = A B^T (complex, M x K and Ncols x K, row-major) through the Ozaki kernels:
// embed both operands, one oz_gemm launch.  skip_stage >= 0 leaves that stage
// unloaded (short wait limit) to exercise the bounded-wait failure path.
int oz_gemm_impl(int M, int Ncols, int K, int slices, const double* A, const double* B, double* C, int skip_stage) {
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return CCSD_ERR_OOM;
    h->cfg.precision = CCSD_OZAKI;
    h->oz_slices = slices;
    h->oz_on = 1;
    h->has_oz = true;
    h->cur_oz = true;
    Alloc al{h};
    auto fail = [&](int code) { ccsd_destroy(h); return code; };
    const long long nA = (long long)M * K, nB = (long long)Ncols * K, nC = (long long)M * Ncols;
    std::vector<double2> hA((size_t)nA), hB((size_t)nB);
    std::memcpy(hA.data(), A, (size_t)nA * 16);
    std::memcpy(hB.data(), B, (size_t)nB * 16);
    h->buf[B_STA] = upload(al, hA, h->st); h->bufsize[B_STA] = nA;
    h->buf[B_STB] = upload(al, hB, h->st); h->bufsize[B_STB] = nB;
    h->buf[B_ZR] = (double2*)al.get((size_t)nC * 16); h->bufsize[B_ZR] = nC;
    h->tc_err = (int*)al.get(sizeof(int));
    if (al.err) return fail(al.err);
    if (cudaMemsetAsync(h->buf[B_ZR], 0, (size_t)nC * 16, h->st) != cudaSuccess ||
        cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    const int kpad = (2 * K + OZ_BK - 1) / OZ_BK * OZ_BK;
    TcBuf ta{}, tb{};
    int rc;
    if ((rc = tc_alloc(h, al, ta, M, kpad)) || (rc = tc_alloc(h, al, tb, 2LL * Ncols, kpad))) return fail(rc);
    if ((rc = add_embed(h, al, B_STA, ta, 0, M, K, {0}, tab({{M, K}}), tab({{K, 1}}), false)) ||
        (rc = add_embed(h, al, B_STB, tb, 1, Ncols, K, {0}, tab({{Ncols, K}}), tab({{K, 1}}), false)))
        return fail(rc);
    std::vector<long long> oc;
    for (int m = 0; m < M; ++m) oc.push_back((long long)m * Ncols);
    if ((rc = add_tc(h, al, ta, tb, B_ZR, M, 2 * Ncols, 1, 1, {0}, {0}, oc, tab({{Ncols, 1}}), 1.0, 1)))
        return fail(rc);
    if (h->oz_work_elems) { h->oz_work = (double2*)al.get((size_t)h->oz_work_elems * 16); if (al.err) return fail(al.err); }
    if (skip_stage >= 0) {
        h->tcs[0].z.skip_stage = skip_stage;
        h->tcs[0].z.spin_limit = 1LL << 14;
    }
    launch_embed(h, h->embeds[0]);
    launch_embed(h, h->embeds[1]);
    launch_tc(h, h->tcs[0]);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    int flag = 0;
    if (cudaMemcpy(&flag, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(C, h->buf[B_ZR], (size_t)nC * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CCSD_ERR_CUDA);
    if (flag) return fail(CCSD_ERR_TIMEOUT);
    ccsd_destroy(h);
    return CCSD_OK;
}

}  // namespace

extern "C" {

int ccsd_oz_gemm(int M, int Ncols, int K, int slices, const double* A, const double* B, double* C) {
    ApiScope api_scope_;
    if (M < 1 || Ncols < 1 || K < 1 || M > 4096 || Ncols > 4096 || K > 8192 || slices < 1 ||
        slices > OZ_MAX_SLICES || !A || !B || !C)
        return CCSD_ERR_INVALID;
    return oz_gemm_impl(M, Ncols, K, slices, A, B, C, -1);
}

int ccsd_oz_timeout_selftest(void) {
    ApiScope api_scope_;
    std::vector<double> a(128 * 64 * 2, 1.0), c(128 * 128 * 2, 0.0);
    return oz_gemm_impl(128, 128, 64, 2, a.data(), a.data(), c.data(), 1);
}

int ccsd_tc_selftest(int M, int Ncols, int K, int nterms, unsigned long long seed, double* rel_err) {
    ApiScope api_scope_;
    if (M < 1 || Ncols < 1 || K < 1 || M > 4096 || Ncols > 4096 || K > 4096 || (nterms != 1 && nterms != 3) || !rel_err)
        return CCSD_ERR_INVALID;
    return tc_selftest_impl(M, Ncols, K, nterms, seed, -1, rel_err);
}

int ccsd_tc_timeout_selftest(void) {
    ApiScope api_scope_;
    double err = 0.0;
    return tc_selftest_impl(128, 128, 64, 1, 1, 1, &err);
}

int ccsd_create(const ccsd_config* cfg, const ccsd_inputs* in, void* stream, ccsd_t* out) {
    ApiScope api_scope_;
    if (!out) return CCSD_ERR_INVALID;
    *out = nullptr;
    if (!valid_cfg(cfg) || !in || (in->int_dtype != CCSD_C128 && in->int_dtype != CCSD_C64)) return CCSD_ERR_INVALID;
    const void* ins[9] = {in->f_oo, in->f_vv, in->f_ov, in->oooo, in->ooov, in->oovv, in->ovvo, in->ovvv, in->vvvv};
    for (const void* p : ins) if (!p) return CCSD_ERR_INVALID;
    bool on_dev[9];
    for (int i = 0; i < 9; ++i) on_dev[i] = is_device_ptr(ins[i]);
    ccsd_ctx* h = new (std::nothrow) ccsd_ctx();
    if (!h) return CCSD_ERR_OOM;
    init_ctx(h, cfg);
    h->st = (cudaStream_t)stream;
    Alloc al{h};
    auto fail = [&](int code) { ccsd_destroy(h); return code; };
    int rc = setup_handle(h, al, ins, on_dev, in->int_dtype, in->vvvv_on_host != 0);
    if (rc) return fail(rc);
    for (int ei : h->const_embeds) launch_embed(h, h->embeds[ei]);
    if (cudaMallocHost(&h->norm_host, sizeof(double)) != cudaSuccess) { cudaGetLastError(); h->norm_host = nullptr; return fail(CCSD_ERR_OOM); }
    if (cudaEventCreateWithFlags(&h->ev_norm, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); h->ev_norm = nullptr; return fail(CCSD_ERR_CUDA); }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    *out = h;
    return CCSD_OK;
}

int ccsd_residual(ccsd_t h, const void* t1, const void* t2, void* r1, void* r2) {
    ApiScope api_scope_;
    if (!h || !t1 || !t2 || !r1 || !r2) return CCSD_ERR_INVALID;
    // the kernels read and write these directly: host memory is refused, not faulted on
    if (!is_device_ptr(t1) || !is_device_ptr(t2) || !is_device_ptr(r1) || !is_device_ptr(r2)) return CCSD_ERR_INVALID;
    h->launches = 0;
    double2* save[4] = {h->buf[B_T1], h->buf[B_T2], h->buf[B_R1], h->buf[B_R2]};
    h->buf[B_T1] = (double2*)t1; h->buf[B_T2] = (double2*)t2;
    h->buf[B_R1] = (double2*)r1; h->buf[B_R2] = (double2*)r2;
    int rc = run_residual(h);
    h->buf[B_T1] = save[0]; h->buf[B_T2] = save[1]; h->buf[B_R1] = save[2]; h->buf[B_R2] = save[3];
    return rc;
}

int ccsd_iterate(ccsd_t h, int n_iter, int* done, double* max_resid) {
    ApiScope api_scope_;
    if (!h || n_iter < 0) return CCSD_ERR_INVALID;
    if (done) *done = 0;
    h->launches = 0;
    for (int it = 0; it < n_iter; ++it) {
        int d = 0;
        double mr = 0.0;
        int rc = iter_begin(h);
        if (rc) return rc;
        rc = iter_end(h, &d, &mr);
        if (max_resid) *max_resid = mr;
        if (rc) return rc;
        if (d) { if (done) *done = 1; return CCSD_OK; }
    }
    CK(cudaStreamSynchronize(h->st));
    return CCSD_OK;
}

int ccsd_solve(ccsd_t h, int* iterations, double* max_resid) {
    ApiScope api_scope_;
    if (!h) return CCSD_ERR_INVALID;
    int done = 0, it = 0;
    double mr = 0.0;
    const bool mixed = h->cfg.precision == CCSD_MIXED;
    const double tol0 = h->cfg.conv_tol;
    if (mixed) {
        if (!h->fp32) ccsd_set_precision(h, CCSD_MIXED);   // keeps the DIIS history of mixed iterations
        h->cfg.conv_tol = std::max(h->cfg.mixed_tol, tol0);
    }
    for (; it <= h->cfg.max_iter; ++it) {
        int rc = ccsd_iterate(h, 1, &done, &mr);
        if (rc) { h->cfg.conv_tol = tol0; if (iterations) *iterations = it; return rc; }
        if (done) break;
    }
    h->cfg.conv_tol = tol0;
    if (mixed && done) {
        // polish (FP64, or the FP64-accurate Ozaki form): the fixed point of the exact equations
        int rc = ccsd_set_precision(h, h->cfg.polish_precision == CCSD_OZAKI ? CCSD_OZAKI : CCSD_FP64);
        if (rc) { if (iterations) *iterations = it; if (max_resid) *max_resid = mr; return rc; }
        int d2 = 0;
        for (int p = 0; p < h->cfg.polish_iters; ++p) {
            rc = ccsd_iterate(h, 1, &d2, &mr);
            if (rc) {
                // the handle goes back to the mixed form; the failure's code and its
                // ccsd_last_error text are what the caller sees
                char why[sizeof g_errbuf];
                memcpy(why, g_errbuf, sizeof why);
                const int back = ccsd_set_precision(h, CCSD_MIXED);
                memcpy(g_errbuf, why, sizeof why);
                if (back) {
                    const size_t n = strlen(g_errbuf);
                    snprintf(g_errbuf + n, sizeof g_errbuf - n, "%s(the handle stayed in the polish precision)",
                             n ? " " : "");
                }
                if (iterations) *iterations = it;
                if (max_resid) *max_resid = mr;
                return rc;
            }
            if (d2) break;
            ++it;
        }
        if ((rc = ccsd_set_precision(h, CCSD_MIXED))) return rc;
    }
    if (iterations) *iterations = it;
    if (max_resid) *max_resid = mr;
    return done ? CCSD_OK : CCSD_ERR_NOT_CONVERGED;
}

int ccsd_set_precision(ccsd_t h, int precision) {
    ApiScope api_scope_;
    if (!h) return CCSD_ERR_INVALID;
    if (precision == CCSD_FP64) { h->fp32 = 0; h->oz_on = 0; }
    else if (precision == CCSD_MIXED && h->cfg.precision == CCSD_MIXED) { h->fp32 = 1; h->oz_on = 0; }
    else if (precision == CCSD_OZAKI && h->has_oz) { h->fp32 = 0; h->oz_on = 1; }
    else return CCSD_ERR_INVALID;
    if (h->d_diis) CK(cudaMemcpyAsync(h->d_diis, &h->diis_init, sizeof(DiisState), cudaMemcpyHostToDevice, h->st));
    return CCSD_OK;
}

int ccsd_energy(ccsd_t h, double* e_real, double* e_imag) {
    ApiScope api_scope_;
    if (!h) return CCSD_ERR_INVALID;
    if (h->in32[B_OOVV])
        energy_partial<<<h->red_blocks, 256, 0, h->st>>>(h->buf[B_T1], h->buf[B_T2], h->buf[B_FOV_IN], h->shadow[B_OOVV],
                                                         h->N, h->o, h->v, h->cred);
    else
        energy_partial<<<h->red_blocks, 256, 0, h->st>>>(h->buf[B_T1], h->buf[B_T2], h->buf[B_FOV_IN], h->buf[B_OOVV],
                                                         h->N, h->o, h->v, h->cred);
    final_csum<<<1, 32, 0, h->st>>>(h->cred, h->red_blocks, h->cred_out);
    double2 e;
    CK(cudaMemcpyAsync(&e, h->cred_out, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (e_real) *e_real = e.x / h->N;
    if (e_imag) *e_imag = e.y / h->N;
    return CCSD_OK;
}

int ccsd_get_amplitudes(ccsd_t h, void* t1, void* t2) {
    ApiScope api_scope_;
    if (!h || !t1 || !t2) return CCSD_ERR_INVALID;
    CK(cudaMemcpyAsync(t1, h->buf[B_T1], (size_t)h->n1 * 16, cudaMemcpyDefault, h->st));
    CK(cudaMemcpyAsync(t2, h->buf[B_T2], (size_t)h->n2 * 16, cudaMemcpyDefault, h->st));
    CK(cudaStreamSynchronize(h->st));
    return CCSD_OK;
}

int ccsd_set_amplitudes(ccsd_t h, const void* t1, const void* t2) {
    ApiScope api_scope_;
    if (!h || !t1 || !t2) return CCSD_ERR_INVALID;
    CK(cudaMemcpyAsync(h->buf[B_T1], t1, (size_t)h->n1 * 16, cudaMemcpyDefault, h->st));
    CK(cudaMemcpyAsync(h->buf[B_T2], t2, (size_t)h->n2 * 16, cudaMemcpyDefault, h->st));
    if (h->d_diis) CK(cudaMemcpyAsync(h->d_diis, &h->diis_init, sizeof(DiisState), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return CCSD_OK;
}

int ccsd_last_launch_count(ccsd_t h, long long* launches) {
    ApiScope api_scope_;
    if (!h || !launches) return CCSD_ERR_INVALID;
    *launches = h->launches;
    return CCSD_OK;
}


int ccsd_trace_enable(ccsd_t h, int enable) {
    ApiScope api_scope_;
    if (!h) return CCSD_ERR_INVALID;
    const size_t n = h->seq.size() + 1;          // plan steps + the amplitude update
    if (enable && h->ev0.empty()) {
        h->ev0.resize(n); h->ev1.resize(n);
        for (size_t i = 0; i < n; ++i) {
            CK(cudaEventCreate(&h->ev0[i]));
            CK(cudaEventCreate(&h->ev1[i]));
        }
    }
    h->step_ms.assign(n, 0.0);
    h->step_calls.assign(n, 0);
    h->trace = enable ? 1 : 0;
    return CCSD_OK;
}

int ccsd_trace_count(ccsd_t h, int* n_steps) {
    ApiScope api_scope_;
    if (!h || !n_steps) return CCSD_ERR_INVALID;
    *n_steps = (int)h->seq.size() + 1;
    return CCSD_OK;
}

int ccsd_trace_step(ccsd_t h, int i, const char** name, long long* calls, double* total_ms,
                    double* flops, double* bytes) {
    ApiScope api_scope_;
    if (!h || i < 0 || i > (int)h->seq.size()) return CCSD_ERR_INVALID;
    const bool upd = i == (int)h->seq.size();
    if (name) *name = upd ? "update" : h->seq[i].name;
    if (calls) *calls = i < (int)h->step_calls.size() ? h->step_calls[i] : 0;
    if (total_ms) *total_ms = i < (int)h->step_ms.size() ? h->step_ms[i] : 0.0;
    if (flops) *flops = upd ? 0.0 : h->seq[i].flops;
    if (bytes) *bytes = upd ? (h->cfg.diis_depth ? 80.0 : 48.0) * (double)(h->n1 + h->n2) : h->seq[i].bytes;
    return CCSD_OK;
}

int ccsd_batch_create(int n, const ccsd_config* cfgs, const ccsd_inputs* inputs, ccsd_batch_t* out) {
    ApiScope api_scope_;
    if (!out || n < 1 || n > 4096 || !cfgs || !inputs) return CCSD_ERR_INVALID;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (cfgs[i].precision != cfgs[0].precision || cfgs[i].diis_depth != cfgs[0].diis_depth ||
            cfgs[i].precision == CCSD_OZAKI || cfgs[i].polish_precision != CCSD_FP64) {
            refuse("batch members share one precision (FP64 or mixed, FP64 polish) and one DIIS depth");
            return CCSD_ERR_INVALID;
        }
    ccsd_batch* B = new (std::nothrow) ccsd_batch();
    if (!B) return CCSD_ERR_OOM;
    B->n = n;
    auto fail = [&](int code) { ccsd_batch_destroy(B); return code; };
    if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); B->st = nullptr; return fail(CCSD_ERR_CUDA); }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); B->fork = nullptr; return fail(CCSD_ERR_CUDA); }
    for (int i = 0; i < n; ++i) {
        ccsd_t h = nullptr;
        int rc = ccsd_create(&cfgs[i], &inputs[i], B->st, &h);
        if (rc) return fail(rc);
        B->m.push_back(h);
    }
    B->fp32 = cfgs[0].precision == CCSD_MIXED ? 1 : 0;
    void* p = nullptr;
    int rc;
    if ((rc = batch_alloc(B, sizeof(double) * n, &p))) return fail(rc);
    B->d_norms = (double*)p;
    if ((rc = batch_alloc(B, sizeof(int) * n, &p))) return fail(rc);
    B->d_done = (int*)p;
    B->done.assign(n, 0);
    if (cudaMemsetAsync(B->d_done, 0, sizeof(int) * n, B->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    // groups of members with equal plan signatures (their members' norms and done flags
    // are contiguous slices of d_norms / d_done)
    std::vector<std::pair<std::vector<std::pair<int, int>>, std::vector<int>>> classes;
    for (int i = 0; i < n; ++i) {
        const auto sig = plan_signature(B->m[i]);
        size_t c = 0;
        while (c < classes.size() && classes[c].first != sig) ++c;
        if (c == classes.size()) classes.push_back({sig, {}});
        classes[c].second.push_back(i);
    }
    // the members are renumbered group by group so that each group's slice is contiguous;
    // `order` maps a slot of d_norms back to the caller's member index
    int slot = 0;
    for (auto& cl : classes) {
        B->groups.emplace_back(new (std::nothrow) Group());
        if (!B->groups.back()) return fail(CCSD_ERR_OOM);
        Group& g = *B->groups.back();
        for (int i : cl.second) { g.m.push_back(B->m[i]); g.ids.push_back(i); }
        if ((rc = group_build(g, B->fp32, {}, B->d_norms + slot, B->d_done + slot, B->st))) return fail(rc);
        slot += (int)cl.second.size();
        cudaStream_t gs = nullptr;
        cudaEvent_t ge = nullptr;
        if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return fail(CCSD_ERR_CUDA); }
        B->gst.push_back(gs);
        if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return fail(CCSD_ERR_CUDA); }
        B->gev.push_back(ge);
    }
    if (cudaStreamSynchronize(B->st) != cudaSuccess) return fail(CCSD_ERR_CUDA);
    *out = B;
    return CCSD_OK;
}

int ccsd_batch_iterate(ccsd_batch_t B, int n_iter, int* done, double* max_resid) {
    ApiScope api_scope_;
    if (!B || n_iter < 0) return CCSD_ERR_INVALID;
    int rc;
    if (!B->tuned) {
        // warm every kernel with one residual of each group, then tune the contractions
        for (auto& g : B->groups) group_residual(*g, B->st);
        CK(cudaStreamSynchronize(B->st));
        if ((rc = batch_autotune(B))) return rc;
    }
    if (!B->graph && (rc = batch_capture(B))) return rc;
    std::vector<double> slots((size_t)B->n, 0.0);
    std::vector<double> norms((size_t)B->n, 0.0);
    for (int it = 0; it < n_iter; ++it) {
        CK(cudaGraphLaunch(B->graph, B->st));
        CK(cudaMemcpyAsync(slots.data(), B->d_norms, sizeof(double) * B->n, cudaMemcpyDeviceToHost, B->st));
        CK(cudaStreamSynchronize(B->st));
        for (auto& g : B->groups) if ((rc = group_check_err(*g, B->st))) return rc;
        // slot order -> member order
        int slot = 0;
        for (auto& g : B->groups) for (int id : g->ids) norms[id] = slots[slot++];
        bool changed = false, all = true;
        for (int i = 0; i < B->n; ++i) {
            if (!std::isfinite(norms[i])) { refuse("a batch member's max|R| is not finite: it diverged"); return CCSD_ERR_DIVERGED; }
            if (!B->done[i] && norms[i] < B->m[i]->cfg.conv_tol) { B->done[i] = 1; changed = true; }
            all = all && B->done[i];
        }
        if (changed) {
            std::vector<int> flags((size_t)B->n);
            slot = 0;
            for (auto& g : B->groups) for (int id : g->ids) flags[slot++] = B->done[id];
            CK(cudaMemcpyAsync(B->d_done, flags.data(), sizeof(int) * B->n, cudaMemcpyHostToDevice, B->st));
            CK(cudaStreamSynchronize(B->st));
        }
        if (all) break;
    }
    for (int i = 0; i < B->n; ++i) {
        if (done) done[i] = B->done[i];
        if (max_resid) max_resid[i] = norms[i];
    }
    return CCSD_OK;
}

int ccsd_batch_energy(ccsd_batch_t B, double* e_real, double* e_imag) {
    ApiScope api_scope_;
    if (!B || !e_real) return CCSD_ERR_INVALID;
    for (int i = 0; i < B->n; ++i) {
        double er = 0.0, ei = 0.0;
        int rc = ccsd_energy(B->m[i], &er, &ei);
        if (rc) return rc;
        e_real[i] = er;
        if (e_imag) e_imag[i] = ei;
    }
    return CCSD_OK;
}

int ccsd_batch_member(ccsd_batch_t B, int i, ccsd_t* h) {
    ApiScope api_scope_;
    if (!B || i < 0 || i >= B->n || !h) return CCSD_ERR_INVALID;
    *h = B->m[i];
    return CCSD_OK;
}

int ccsd_batch_stats(ccsd_batch_t B, long long* launches_per_iteration, int* tile_cfgs, int max_cfgs) {
    ApiScope api_scope_;
    if (!B) return CCSD_ERR_INVALID;
    if (launches_per_iteration) {
        long long n = 0;
        for (auto& g : B->groups) n += group_launches(*g, true);
        *launches_per_iteration = n;
    }
    if (tile_cfgs) {
        int k = 0;
        for (auto& g : B->groups)
            for (const BatchGroup& bg : g->gemms) if (k < max_cfgs) tile_cfgs[k++] = bg.cfg;
    }
    return CCSD_OK;
}

int ccsd_batch_destroy(ccsd_batch_t B) {
    ApiScope api_scope_;
    if (!B) return CCSD_ERR_INVALID;
    if (B->st) cudaStreamSynchronize(B->st);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (auto& g : B->groups) if (g) group_free(*g);
    for (ccsd_ctx* h : B->m) ccsd_destroy(h);
    for (void* p : B->owned) cudaFree(p);
    for (cudaStream_t s : B->gst) cudaStreamDestroy(s);
    for (cudaEvent_t e : B->gev) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->st) cudaStreamDestroy(B->st);
    delete B;
    return CCSD_OK;
}

namespace {

void server_release(ccsd_server* S) {
    for (Lane& L : S->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        for (cudaStream_t g : L.gst) cudaStreamDestroy(g);
        for (cudaEvent_t e : L.gev) cudaEventDestroy(e);
        if (L.done) cudaEventDestroy(L.done);
        if (L.fork) cudaEventDestroy(L.fork);
        if (L.h_norms) cudaFreeHost(L.h_norms);
        if (L.st) {
            // the caller's stream waits for everything the lane did
            cudaEvent_t e = nullptr;
            if (S->st && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, L.st);
                cudaStreamWaitEvent(S->st, e, 0);
                cudaEventDestroy(e);
            }
            cudaStreamDestroy(L.st);
        }
        L = Lane();
    }
    if (S->start) cudaEventDestroy(S->start);
    if (S->own_stream && S->st) cudaStreamDestroy(S->st);
    cudaGetLastError();
}

}  // namespace

int ccsd_server_create(size_t hbm_budget_bytes, int max_slots, void* stream, ccsd_server_t* out) {
    ApiScope api_scope_;
    if (!out || max_slots < 1 || max_slots > 1024 || hbm_budget_bytes == 0) return CCSD_ERR_INVALID;
    ccsd_server* S = new (std::nothrow) ccsd_server();
    if (!S) return CCSD_ERR_OOM;
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->t0 = std::chrono::steady_clock::now();
    auto fail = [&](int code) { server_release(S); delete S; return code; };
    if (cudaGetDevice(&S->device) != cudaSuccess) { cudaGetLastError(); return fail(CCSD_ERR_CUDA); }
    S->st = (cudaStream_t)stream;
    if (!S->st) {
        if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); S->st = nullptr; return fail(CCSD_ERR_CUDA); }
        S->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&S->start, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); S->start = nullptr; return fail(CCSD_ERR_CUDA); }
    if (cudaEventRecord(S->start, S->st) != cudaSuccess) { cudaGetLastError(); return fail(CCSD_ERR_CUDA); }
    for (Lane& L : S->lanes) {
        if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); L.st = nullptr; return fail(CCSD_ERR_CUDA); }
        if (cudaStreamWaitEvent(L.st, S->start, 0) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return fail(CCSD_ERR_CUDA); }
        if (cudaMallocHost(&L.h_norms, sizeof(double) * max_slots) != cudaSuccess) { cudaGetLastError(); L.h_norms = nullptr; return fail(CCSD_ERR_OOM); }
    }
    try {
        S->th = std::thread(server_loop, S);
    } catch (...) {
        return fail(CCSD_ERR_OOM);
    }
    *out = S;
    return CCSD_OK;
}

int ccsd_submit(ccsd_server_t S, const ccsd_config* cfg, const ccsd_inputs* in, uint64_t* request_id) {
    ApiScope api_scope_;
    if (!S || !cfg || !in || !request_id || !valid_cfg(cfg) || (in->int_dtype != CCSD_C128 && in->int_dtype != CCSD_C64))
        return CCSD_ERR_INVALID;
    const size_t bytes = request_bytes(*cfg, *in);
    if (!bytes) return CCSD_ERR_INVALID;
    ServerReq* r = new (std::nothrow) ServerReq();
    if (!r) return CCSD_ERR_OOM;
    r->cfg = *cfg;
    r->in = *in;
    r->bytes = bytes;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop) { delete r; return CCSD_ERR_INVALID; }
        r->id = S->next_id++;
        r->t_submit = server_now(S);
        S->all[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv.notify_one();
    *request_id = r->id;
    return CCSD_OK;
}

int ccsd_poll(ccsd_server_t S, uint64_t id, int* state, double* e_corr, double* t_converge_s, int* iterations) {
    ApiScope api_scope_;
    if (!S) return CCSD_ERR_INVALID;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return CCSD_ERR_INVALID;
    const ServerReq* r = it->second;
    if (state) *state = r->state;
    if (e_corr) *e_corr = r->e_re;
    if (t_converge_s) *t_converge_s = (r->state == 2 || r->state < 0) ? r->t_done - r->t_submit : 0.0;
    if (iterations) *iterations = r->iters;
    return CCSD_OK;
}

int ccsd_server_stats(ccsd_server_t S, int* active, int* queued, size_t* admitted_bytes) {
    ApiScope api_scope_;
    if (!S) return CCSD_ERR_INVALID;
    std::lock_guard<std::mutex> lock(S->mu);
    if (active) *active = (int)S->active.size();
    if (queued) *queued = (int)S->pending.size();
    if (admitted_bytes) *admitted_bytes = S->used;
    return CCSD_OK;
}

int ccsd_server_profile(ccsd_server_t S, long long* rounds, long long* group_builds, double* round_seconds,
                        double* build_seconds, double* mean_wait_s, double* mean_run_s) {
    ApiScope api_scope_;
    if (!S) return CCSD_ERR_INVALID;
    std::lock_guard<std::mutex> lock(S->mu);
    if (rounds) *rounds = S->rounds;
    if (group_builds) *group_builds = S->rebuilds;
    if (round_seconds) *round_seconds = S->round_s;
    if (build_seconds) *build_seconds = S->rebuild_s;
    if (mean_wait_s) *mean_wait_s = S->finished ? S->wait_s / (double)S->finished : 0.0;
    if (mean_run_s) *mean_run_s = S->finished ? S->run_s / (double)S->finished : 0.0;
    return CCSD_OK;
}

int ccsd_server_destroy(ccsd_server_t S) {
    ApiScope api_scope_;
    if (!S) return CCSD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_one();
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->all) delete kv.second;
    server_release(S);
    delete S;
    return CCSD_OK;
}

int ccsd_destroy(ccsd_t h) {
    ApiScope api_scope_;
    if (!h) return CCSD_ERR_INVALID;
    if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
    for (void* p : h->owned) cudaFree(p);
    for (cudaEvent_t e : h->ev0) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev1) cudaEventDestroy(e);
    if (h->norm_host) cudaFreeHost(h->norm_host);
    if (h->ev_norm) cudaEventDestroy(h->ev_norm);
    if (h->host_registered) host_unregister(h->host_registered);
    delete h;
    return CCSD_OK;
}

const char* ccsd_last_error(void) { return g_errbuf; }

const char* ccsd_strerror(int code) {
    switch (code) {
        case CCSD_OK: return "ok";
        case CCSD_ERR_INVALID: return "invalid argument (shape, null pointer, dtype or config)";
        case CCSD_ERR_OOM: return "device memory exhausted or admission refused";
        case CCSD_ERR_CUDA: return "CUDA runtime error";
        case CCSD_ERR_NOT_CONVERGED: return "iteration limit reached before convergence";
        case CCSD_ERR_DIVERGED: return "non-finite or diverging residual";
        case CCSD_ERR_TIMEOUT: return "bounded device wait gave up";
        default: return "unknown error code";
    }
}

}  // extern "C"
