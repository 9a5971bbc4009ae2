/*
 * ccsd.h -- C ABI of the GB300 library for periodic spin-orbital CCSD
 * (Yamashita, Kosugi, Matsushita, Sakurai, "A Parallel Computing Method for
 * the Coupled-Cluster Singles and Doubles", arXiv:1911.00242).
 *
 * The library evaluates the T1/T2 residuals of the paper's Eqs. (ori_EqSingle)
 * and (ori_EqDouble) -- equivalently the rearranged Eqs. (EqSingle) and
 * (EqDouble) of Sec. 3.3 -- and performs the amplitude update of Sec. 4.4 on
 * one GPU.  The paper's N_k^2 process grid (Sec. 3.1-3.2) becomes the batch
 * index of grouped complex GEMM kernels.
 *
 * Data layout (row-major, last index fastest, complex = interleaved re,im):
 *   k point: integer triple (k1,k2,k3), 0 <= kd < nd, flat index
 *            (k1*n2 + k2)*n3 + k3; momentum sums are componentwise mod nd
 *            (paper Sec. 3.2.5).  N = n1*n2*n3.
 *   f_oo[k][i][j], f_vv[k][a][b], f_ov[k][i][a]   Fock blocks, complex128,
 *            f_ov[k][i][a] = <i k|f|a k>                        (Sec. 2)
 *   B[kp][kq][kr][p][q][r][s]  antisymmetrized integrals <p kp q kq||r kr s ks>
 *            with ks = kp + kq - kr, for B in oooo, ooov, oovv, ovvo, ovvv,
 *            vvvv (every other class follows from the symmetries of Sec. 3.3)
 *   t1[k][i][a], t2[ki][kj][ka][i][j][a][b] (kb = ki + kj - ka), complex128
 *
 * Errors: every entry point returns 0 (CCSD_OK) or a negative CCSD_ERR_* code;
 * ccsd_strerror() names it.  No exception crosses the ABI.  After a
 * CCSD_ERR_CUDA the handle should be destroyed.
 * Threading: one handle must not be used from two host threads at once.  All
 * device work is enqueued on the stream given at creation; calls that return
 * host scalars synchronize that stream.
 */
#ifndef CCSD_GB300_H
#define CCSD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCSD_OK                 0
#define CCSD_ERR_INVALID      (-1)  /* bad shape, null pointer, dtype, config   */
#define CCSD_ERR_OOM          (-2)  /* device allocation or admission refused   */
#define CCSD_ERR_CUDA         (-3)  /* a CUDA runtime call failed               */
#define CCSD_ERR_NOT_CONVERGED (-4) /* max_iter reached; results still readable */
#define CCSD_ERR_DIVERGED     (-5)  /* non-finite residual                       */
#define CCSD_ERR_TIMEOUT      (-6)  /* a bounded device wait gave up             */

#define CCSD_FP64   0   /* every contraction in FP64 (DFMA)                    */
#define CCSD_MIXED  1   /* contractions in FP32 arithmetic with FP32 accumulation
                           (operands rounded from the FP64 data); update, norms,
                           DIIS and energy stay FP64; ccsd_solve finishes with
                           polish_iters FP64 iterations                       */

#define CCSD_OZAKI  2   /* FP64-accurate: the ladder, ring and hole-hole
                           contractions on the BF16 tensor cores by the Ozaki
                           scheme (error-free splitting of each operand row
                           into oz_slices 7-bit slices under a power-of-two
                           scale; slice products summed exactly in TMEM, then
                           in double-float), everything else in FP64 (DFMA).
                           Relative error of a contraction about
                           2^-(7 oz_slices) of sum |a||b| (7 slices: FP64-like);
                           operand rows must lie within about 1e-36 .. 1e36;
                           nvir <= 96 (one W' row is staged in shared memory);
                           the other GEMMs run in double-float (about 48 bits)  */

#define CCSD_C128   0   /* integral blocks complex128                          */
#define CCSD_C64    1   /* integral blocks complex64 (Fock blocks stay complex128):
                           the FP64 form widens every element exactly to double on
                           load, so it solves the equations of exactly these values;
                           the mixed form reads them as stored                    */

typedef struct ccsd_ctx* ccsd_t;

typedef struct {
    int    nk_dims[3];    /* k grid (n1, n2, n3), each >= 1                     */
    int    nocc, nvir;    /* occupied / virtual spin orbitals per k, >= 1       */
    int    precision;     /* CCSD_FP64, CCSD_MIXED or CCSD_OZAKI                */
    int    diis_depth;    /* 0 = plain successive substitution (paper Sec. 4.4.18);
                             2..8 = Pulay DIIS over that many updates            */
    int    max_iter;      /* used by ccsd_solve, >= 0                           */
    double conv_tol;      /* max|R1| and max|R2| threshold, Eqs. (criterion_single,
                             criterion_double); finite, >= 0 (0: never met)      */
    int    polish_iters;  /* CCSD_MIXED: polish iterations ccsd_solve runs after the
                             mixed ones (0..100)                                 */
    double mixed_tol;     /* CCSD_MIXED: ccsd_solve switches to FP64 once the mixed
                             max|R| < max(mixed_tol, conv_tol); finite, >= 0    */
    int    lean;          /* work-memory policy.  0: automatic -- problems whose
                             tensor-core operands would exceed 24 GB share two
                             operand buffers rewritten every residual, and the
                             ladder's W' is formed in slabs of at most 12 GB;
                             1: that lean layout at any size, with the W' slabs
                             and the tensor-core ladder chunks cut to about a
                             third (same results, more launches)                */
    int    oz_slices;     /* CCSD_OZAKI: slices per operand, 3..8 (0 = 7)       */
    int    polish_precision; /* CCSD_MIXED: arithmetic of the polish iterations,
                             CCSD_FP64 (default, 0) or CCSD_OZAKI (the handle then
                             also carries the Ozaki steps; their operands share
                             the pooled buffers in the lean layout)             */
} ccsd_config;

typedef struct {
    /* Fock blocks and the six integral blocks in the layout above.  Each
     * pointer may be device memory (borrowed: it must stay valid and unchanged
     * until ccsd_destroy) or host memory (copied into library-owned device
     * memory during ccsd_create; pinned host memory copies fastest). */
    const void *f_oo, *f_vv, *f_ov;
    const void *oooo, *ooov, *oovv, *ovvo, *ovvv, *vvvv;
    int int_dtype;        /* CCSD_C128 or CCSD_C64 (the six integral blocks)    */
    int vvvv_on_host;     /* 1: a host vvvv stays in host memory and the kernels
                             read it in place (the library registers it as
                             mapped pinned memory unless the caller already
                             did, and unregisters it when the last handle
                             reading it is destroyed); it is read once per
                             iteration (the ladder's W' formation), so this frees
                             its N^3 v^4 elements of device memory for about one
                             host-link transfer of it per iteration.  0:
                             host inputs are copied.  Ignored for a device
                             pointer.  */
} ccsd_inputs;

/* Creates a solver for one problem.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream) on the current device.  The amplitudes start at zero,
 * so the first update produces t0 = f(0) (paper Sec. 3.2.2).  Allocates all
 * work memory up front; returns CCSD_ERR_OOM if it does not fit. */
int ccsd_create(const ccsd_config* cfg, const ccsd_inputs* in, void* stream, ccsd_t* out);

/* Bytes of device memory ccsd_create allocates for this config when
 * `inputs_on_device` is 1 (borrowed inputs) or 0 (copied inputs) and the
 * integral blocks are int_dtype (CCSD_C128 / CCSD_C64): the total of a dry run
 * of its allocations and plan, nothing allocated.  CCSD_ERR_INVALID for a bad
 * config or dtype. */
int ccsd_footprint(const ccsd_config* cfg, int inputs_on_device, int int_dtype, size_t* bytes);

/* Builds the launch plan of this config on the host only (no GPU, no device
 * memory) and checks that every element each launch can touch lies inside
 * its buffer.  *n_launches receives the kernel launches of one residual
 * evaluation, *table_bytes the size of the plan's index tables. */
int ccsd_plan_check(const ccsd_config* cfg, long long* n_launches, size_t* table_bytes);

/* The launch plan of this config, built on the host as ccsd_plan_check does: for
 * each of its *n_steps steps (at most max_steps are written; arrays may be NULL)
 * the step kind (0 FP64/FP32 GEMM, 1 copy, 2 permutation, 3 tau, 4 antisymmetrize,
 * 5 tensor-core operand embedding, 6 tensor-core GEMM, 7 zero, 9 complex64 copy,
 * 10 W' formation, 11 fused Fock terms, 12 transposed F'vv, 13 fused double-float
 * Fock terms, 14 their double-float copies), the iterations it
 * runs in (mode 0 all; 1 without tensor cores; 2 split-TF32 tensor-core steps of
 * mixed iterations; 3 mixed iterations only; 4 all but mixed iterations; 5 Ozaki
 * iterations only), its algorithmic real flops and its
 * name (static strings owned by the library). */
int ccsd_plan_describe(const ccsd_config* cfg, int max_steps, int* kinds, int* modes, double* flops,
                       const char** names, int* n_steps);

/* Self-test of the tensor-core GEMM of the mixed form: C = A B^T for random
 * complex A (M x K) and B (Ncols x K) through the TF32 path (nterms 1: plain
 * TF32, 3: split TF32) against the FP64 engine; *rel_err = max|dC| / max|C|.
 * Sizes up to 4096.  CCSD_ERR_TIMEOUT if a bounded device wait gave up. */
int ccsd_tc_selftest(int M, int Ncols, int K, int nterms, unsigned long long seed, double* rel_err);

/* Failure-detection self-test of the tensor-core GEMM: a 128 x 128 x 64 product
 * in which the loader never fills one pipeline stage, with a short wait limit,
 * so the MMA issuer's bounded wait gives up.  The kernel records the timeout in
 * its error word, stops issuing, drains its copies and MMAs in flight, frees its
 * TMEM and returns; the call returns CCSD_ERR_TIMEOUT (the expected outcome) and
 * the CUDA context stays usable.  Any other code means the failure path is broken. */
int ccsd_tc_timeout_selftest(void);

/* The Ozaki-scheme GEMM of CCSD_OZAKI on its own: C = A B^T for complex A
 * (M x K) and B (Ncols x K), row-major, complex interleaved, all host arrays
 * (C is overwritten), with `slices` BF16 slices per operand row (1..8).  The
 * operands are split and multiplied by exactly the kernels the solver runs;
 * tests compare C with an FP64 product on the host.  Sizes M, Ncols up to 4096,
 * K up to 8192.  CCSD_ERR_TIMEOUT if a bounded device wait gave up. */
int ccsd_oz_gemm(int M, int Ncols, int K, int slices, const double* A, const double* B, double* C);

/* Failure-detection self-test of the Ozaki GEMM, as ccsd_tc_timeout_selftest (here
 * the loader never fills one pair of A-slice stages): returns CCSD_ERR_TIMEOUT when
 * the failure path works. */
int ccsd_oz_timeout_selftest(void);

/* One residual evaluation R(t) (paper Eqs. ori_EqSingle, ori_EqDouble with the
 * full Fock matrix inside F~): t1, t2 are read and r1, r2 written, all device
 * pointers in the layout above (r1 like t1, r2 like t2).  Does not touch the
 * handle's amplitudes.  CCSD_ERR_INVALID if a pointer is not device (or
 * managed) memory. */
int ccsd_residual(ccsd_t h, const void* t1, const void* t2, void* r1, void* r2);

/* Up to n_iter iterations on the handle's amplitudes.  Each computes R(t);
 * if max(max|R1|, max|R2|) < conv_tol it sets *done = 1 and stops without
 * updating; otherwise t <- t + R/D (paper Sec. 4.4.19, D from the Fock
 * diagonal), followed by DIIS extrapolation when diis_depth > 0 (history, Gram
 * matrix and Pulay solve in device memory; an iteration whose DIIS system is
 * singular keeps the plain update).  The only host synchronization of an iteration
 * is the read of max|R|.  *max_resid receives the last max|R| (may be NULL).
 * Returns CCSD_ERR_DIVERGED if R is not finite. */
int ccsd_iterate(ccsd_t h, int n_iter, int* done, double* max_resid);

/* Iterates until convergence or cfg->max_iter updates; CCSD_ERR_NOT_CONVERGED
 * when the limit is reached (the amplitudes remain readable).  For CCSD_MIXED
 * handles: mixed iterations until max|R| < max(mixed_tol, conv_tol), then up
 * to polish_iters polish iterations in polish_precision (fewer if their
 * max|R| < conv_tol);
 * CCSD_OK when the mixed phase reached its tolerance. */
int ccsd_solve(ccsd_t h, int* iterations, double* max_resid);

/* Arithmetic of the following ccsd_iterate/ccsd_residual calls: CCSD_FP64 on
 * any handle, CCSD_MIXED only on handles created with it, CCSD_OZAKI on
 * handles created with it or with CCSD_MIXED and polish_precision =
 * CCSD_OZAKI.  Clears the DIIS history. */
int ccsd_set_precision(ccsd_t h, int precision);

/* Correlation energy of the current amplitudes per unit cell (supercell
 * total / N_k): sum f_ia t_i^a + 1/4 sum <ij||ab> t_ij^ab
 * + 1/2 sum <ij||ab> t_i^a t_j^b.  The paper states no energy expression; this
 * is the standard spin-orbital one.  e_imag is zero for time-reversal
 * symmetric inputs. */
int ccsd_energy(ccsd_t h, double* e_real, double* e_imag);

/* Copy the amplitudes out of / into the handle; host or device pointers. */
int ccsd_get_amplitudes(ccsd_t h, void* t1, void* t2);
int ccsd_set_amplitudes(ccsd_t h, const void* t1, const void* t2);

/* Number of kernel launches the last ccsd_iterate/ccsd_residual call made. */
int ccsd_last_launch_count(ccsd_t h, long long* launches);

/* Tracing: with tracing enabled, every step of the residual plan and the
 * amplitude update are bracketed by CUDA events on the handle's stream and
 * their durations accumulate per step (enabling resets the accumulators).
 * Steps are numbered 0 .. n_steps-1 in launch order; the last is the update.
 * For step i: its name, how often it ran, total milliseconds, algorithmic real
 * flops per launch (a complex multiply-add counts 8) and algorithmic bytes per
 * launch for the memory-bound steps (0 when not applicable). */
int ccsd_trace_enable(ccsd_t h, int enable);
int ccsd_trace_count(ccsd_t h, int* n_steps);
int ccsd_trace_step(ccsd_t h, int i, const char** name, long long* calls, double* total_ms,
                    double* flops, double* bytes);

/* Waits for the handle's stream, then frees everything the handle owns: its
 * device memory (amplitudes, residuals, work buffers, copied inputs, plan
 * tables), events and pinned buffers, and its count on a host vvvv registration.
 * Borrowed inputs are left untouched.  CCSD_ERR_INVALID for NULL. */
int ccsd_destroy(ccsd_t h);

/* ---------------------------------------------------------------- batched form
 * n independent problems (any mix of grids and orbital counts; one precision,
 * CCSD_FP64 or CCSD_MIXED, and one diis_depth) iterate together on a stream the
 * batch owns.  Members whose plans have the same step sequence form a group; every
 * step of a group's iteration is one grouped launch over its members (contractions
 * in a persistent grouped kernel whose tile shape an autotuner picks on the first
 * iteration; tensor-core contractions, elementwise steps, norms and updates in one
 * launch each), and the groups run concurrently.  An iteration -- residuals,
 * per-member max|R|, update of the members not yet converged, DIIS extrapolation
 * with its history, Gram matrix and Pulay solve kept in device memory -- is
 * replayed as one CUDA graph.  Members stop updating once their max|R| < conv_tol.
 * The problem data follow the rules of ccsd_create (device inputs borrowed).  Each
 * member extrapolates with its own handle's DIIS history, as ccsd_iterate does. */
typedef struct ccsd_batch* ccsd_batch_t;
int ccsd_batch_create(int n, const ccsd_config* cfgs, const ccsd_inputs* inputs, ccsd_batch_t* out);
/* Up to n_iter iterations; done[i] / max_resid[i] per member (arrays of n, may be NULL). */
int ccsd_batch_iterate(ccsd_batch_t b, int n_iter, int* done, double* max_resid);
/* Per-member correlation energy per unit cell (arrays of n; e_imag may be NULL). */
int ccsd_batch_energy(ccsd_batch_t b, double* e_real, double* e_imag);
/* Handle of member i (owned by the batch; usable with ccsd_get_amplitudes etc.). */
int ccsd_batch_member(ccsd_batch_t b, int i, ccsd_t* h);
/* Kernel launches per iteration and the autotuned tile shape of each grouped step. */
int ccsd_batch_stats(ccsd_batch_t b, long long* launches_per_iteration, int* tile_cfgs, int max_cfgs);
/* Destroys every member handle and the batch's graphs, buffers and stream. */
int ccsd_batch_destroy(ccsd_batch_t b);

/* ---------------------------------------------------------------- serving form
 * A request loop on its own host thread.  Submitted solves wait in FIFO order
 * until their device-memory footprint fits in hbm_budget_bytes and one of
 * max_slots slots is free; each admitted solve gets a handle whose integrals and
 * amplitudes stay resident until it finishes.  Admitted solves advance in rounds,
 * one iteration each per round, in lanes by the order of magnitude of their
 * iteration's work: every lane has a stream of its own and runs its rounds at its own
 * pace, so small solves do not wait for the iterations of large ones.  Within a
 * lane's round, solves with the same plan signature, arithmetic and contraction tile
 * shapes form a group, and every step of their residual is one grouped launch (the
 * groups run concurrently); all max|R| come back in one copy, each solve takes its
 * convergence test, and one grouped update (with DIIS) advances the solves that go
 * on.  A solve's iterates are bitwise those it has alone.  Converged solves retire
 * and free their memory for the queue.  A solve runs like ccsd_solve (mixed
 * iterations, then polish_iters iterations in polish_precision, for CCSD_MIXED).
 * The inputs a request points to must stay valid until it is done (host inputs
 * are copied when the request is admitted). */
typedef struct ccsd_server* ccsd_server_t;
/* Starts the loop on the current device: hbm_budget_bytes > 0, 1 <= max_slots <= 1024.
 * `stream` (a cudaStream_t; NULL: the server creates a non-blocking stream of its
 * own) orders the server with the caller's work: the lanes start after the work
 * queued on it before this call, and it waits for the lanes' work when the server
 * is destroyed.  A given stream must outlive the server. */
int ccsd_server_create(size_t hbm_budget_bytes, int max_slots, void* stream, ccsd_server_t* out);
/* Queues one solve (config and input pointers are copied into the request; the
 * data they point to is not) and returns its id.  CCSD_ERR_INVALID for a bad
 * config or after ccsd_server_destroy began. */
int ccsd_submit(ccsd_server_t s, const ccsd_config* cfg, const ccsd_inputs* in, uint64_t* request_id);
/* state: 0 queued, 1 running, 2 done, < 0 the CCSD_ERR_* code it ended with
 * (CCSD_ERR_OOM: larger than the whole budget).  e_corr: energy per unit cell
 * (done only); t_converge_s: submission to completion (finished only). */
int ccsd_poll(ccsd_server_t s, uint64_t id, int* state, double* e_corr, double* t_converge_s, int* iterations);
/* Running solves, queued solves and the device bytes admitted solves hold. */
int ccsd_server_stats(ccsd_server_t s, int* active, int* queued, size_t* admitted_bytes);
/* Statistics of the loop so far: rounds run (over all lanes), groups built (a group
 * is rebuilt when its solves change), the host seconds spent in rounds and, within
 * them, in building groups, and over the admitted solves that finished the mean wait
 * from submission to admission and the mean time from admission to completion.  Any
 * pointer may be NULL.  The paper has no counterpart. */
int ccsd_server_profile(ccsd_server_t s, long long* rounds, long long* group_builds, double* round_seconds,
                        double* build_seconds, double* mean_wait_s, double* mean_run_s);
/* Finishes the admitted solves, cancels the queued ones, joins the thread. */
int ccsd_server_destroy(ccsd_server_t s);

/* The FP64 rate of the current device, measured: the roofline denominator of the
 * FP64 form.  The paper has no counterpart; it states no hardware.  Runs two probe
 * kernels with no memory traffic in their loops -- fused multiply-add chains
 * (DFMA) and FP64 mma.sync (m8n8k4) -- at 2, 4 and 8 blocks of 256 threads per SM,
 * times each with CUDA events on a stream of its own (about 1 s in total, after a
 * warm-up launch per shape) and returns the best rate of each in TFLOP/s (2 flops
 * per multiply-add).  Either pointer may be NULL (that probe is skipped), not both.
 * Synchronizes the device's work it enqueued; allocates 8 bytes of device memory
 * while it runs. */
int ccsd_fp64_peak_probe(double* dfma_tflops, double* dmma_tflops);

/* A static description of a CCSD_* code. */
const char* ccsd_strerror(int code);

/* Why the most recent failing call on this host thread failed, where the library
 * knows more than the code says (an invalid config field, a 32-bit table limit, the
 * CUDA error text, a timed-out device wait); "" if nothing was recorded.  Every
 * entry point but ccsd_energy_noalloc and ccsd_fp64_peak_probe clears it when
 * called from outside the library.  The pointer stays valid for the thread's lifetime. */
const char* ccsd_last_error(void);

/* Correlation energy per unit cell of the amplitudes t1, t2 (same expression
 * as ccsd_energy), for callers that cannot allocate device memory: code
 * running inside a CUDA stream capture, hosts whose allocator owns all device
 * memory, loops that must not pay for an allocation.  The paper has no
 * counterpart; this is a library convenience.
 *   nk_dims, nocc, nvir  problem shape as in ccsd_config
 *   f_ov, oovv, t1, t2   device pointers in the layout above (complex128)
 *   e_out                device pointer to 2 doubles: real, imaginary part
 *   stream               cudaStream_t the work is enqueued on (asynchronous)
 * It allocates nothing: its scratch (one partial sum per momentum block) is a
 * fixed 512 KiB device array inside the library, which every GPU that loads
 * the library keeps until the process exits.  Requires N_k^3 + 1 <= 32768
 * (N_k <= 31); larger grids return CCSD_ERR_INVALID before any launch.  The
 * first call on a device looks the array's device address up once, so make
 * that first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams, or different host
 * threads on one device) race and must be serialized by the caller. */
int ccsd_energy_noalloc(const int nk_dims[3], int nocc, int nvir, const void* f_ov, const void* oovv,
                        const void* t1, const void* t2, void* e_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CCSD_GB300_H */
