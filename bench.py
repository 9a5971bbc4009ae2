"""Benchmark: periodic CCSD amplitude iterations on one GB300 (or N replicas).

Workload (default): the FP64 3D workload -- 2x2x2 k grid (N_k = 8), 8 occupied
and 32 virtual spin orbitals per k, complex128 integrals (vvvv block 8.6 GB),
DIIS(6), seeded synthetic supercell integrals.  One step = one CCSD iteration:
residual R(t) (all contractions), convergence test, update t + R/D, DIIS
extrapolation.  value = iterations per second over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the paper has no code to run) on the
host cores, each step one oracle iteration of the same workload.
Under torchrun every rank solves its own replica (no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ccsd_synth as cs  # noqa: E402

WORKLOADS = {"grid222_o8_v32": dict(diis_depth=6),
             # 2x2x1 grid, same orbitals: the profiling case (vvvv 1.1 GB, still larger than L2)
             "grid221_o8_v32": dict(diis_depth=6),
             # 64 independent problems of uneven size in grouped launches (batched form)
             "batch64": dict(diis_depth=0),
             # Poisson request stream into the serving loop (serving form)
             "serve": dict(diis_depth=6),
             # the mixed-precision workload: 3x3x3 grid, o 8, v 24, complex64 integrals (vvvv 52 GB)
             "grid333_o8_v24_c64": dict(diis_depth=6)}
METRIC = "CCSD iter/s"
TF32_NOMINAL_RATIO = 1.1 / 2.25   # nominal dense TF32 / BF16 tensor rates
SOLVE_TOL = 1e-9                 # max|R| for the time-to-solution comparison


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


def flops_per_iteration(spec):
    N, o, v = spec.nk, spec.nocc, spec.nvir
    # nominal count (complex MAC = 8 real flops): ladder N^4 o^2 v^4, ring 2 N^4 o^3 v^3,
    # hole-hole 2 N^4 o^4 v^2
    return 8.0 * (N ** 4) * (o * o * v ** 4 + 2 * o ** 3 * v ** 3 + 2 * o ** 4 * v * v)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_traffic(kernel_name):
    """DRAM bytes per launch from a committed ncu capture, if it matches the current kernel source."""
    try:
        d = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    import hashlib
    src = open(os.path.join(ROOT, "paper_1911_00242_gb300", "csrc", "zgemm_kb.cuh"), "rb").read()
    if d.get("kernel_source_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return d.get("steps", {}).get(kernel_name)


def fp64_peak(local):
    """The FP64 rate of this GPU, measured by the library's probe (DFMA chains and FP64
    mma.sync, best of several occupancies), with the SM clocks sampled while it runs."""
    import ctypes
    from paper_1911_00242_gb300 import binding
    lib = binding.load()
    clocks = ClockSampler(local)
    clocks.start()
    dfma, dmma = ctypes.c_double(0.0), ctypes.c_double(0.0)
    binding.check(lib.ccsd_fp64_peak_probe(ctypes.byref(dfma), ctypes.byref(dmma)), "ccsd_fp64_peak_probe")
    clk = clocks.stop()
    return {"dfma_tflops": dfma.value, "dmma_tflops": dmma.value, "tflops": max(dfma.value, dmma.value),
            "clocks": clk}


def max_over_ranks(x, dist, device):
    """The slowest rank's value (the job's time); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_iteration(name, seed=41):
    """Seconds of one full oracle iteration of workload `name` on this host's cores: the
    form-A residual (paper Sec. 2) at random antisymmetric amplitudes, the Jacobi update
    t + R/D and the energy (Sec. 4.4), exactly as the oracle computes them."""
    from oracle import ccsd_k, driver
    spec = cs.spec_for(name)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))
    t1, t2 = cs.random_amplitudes(spec, seed)
    D1, D2 = driver.denominators(P)
    t0 = time.perf_counter()
    R1, R2 = ccsd_k.residual(P, t1, t2)
    t1 = t1 + R1 / D1
    t2 = t2 + R2 / D2
    ccsd_k.energy(P, t1, t2)
    secs = time.perf_counter() - t0
    return secs, ("one full oracle iteration of %s itself: form-A residual at random amplitudes, "
                  "Jacobi update, energy (numpy + BLAS on the host cores), %.1f s" % (name, secs))


def run_reference(args, spec):
    """Reference arm: the CPU oracle (the paper ships no code) on this host's cores.

    The K timed steps together are ONE complete oracle iteration of the workload itself,
    formed block by block by the block oracle (form A, paper Sec. 2): the first step forms
    F~ at every k and R1 at every k, every step forms its share of the N_k^3 R2 blocks
    (each intermediate is formed once and shared by the steps), and the last step applies
    the Jacobi update t + R/D and evaluates the energy (Sec. 4.4).  Nothing is scaled:
    value = 1 iteration / the timed seconds, ms_per_step = those seconds / K.  Each warm-up
    step forms one R2 block on a separate oracle object (it pages the inputs in)."""
    import numpy as np
    from oracle import ccsd_k, driver
    from oracle.ccsd_k_block import BlockProblem, BlockResidual
    inp = cs.generate(spec)
    t1, t2 = cs.random_amplitudes(spec, 41)
    BP = BlockProblem(spec.grid, spec.nocc, spec.nvir, inp)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    D1, D2 = driver.denominators(P)
    N = spec.nk
    blocks = [(ki, kj, ka) for ki in range(N) for kj in range(N) for ka in range(N)]
    for w in range(args.warmup):
        BlockResidual(BP, t1, t2).r2(*blocks[(37 * w) % len(blocks)])
    K = args.steps
    parts = np.array_split(np.arange(len(blocks)), K)
    B = BlockResidual(BP, t1, t2)
    R1 = None
    R2 = np.empty_like(t2)
    t0 = time.perf_counter()
    for si in range(K):
        if si == 0:
            B.fock()
            R1 = np.stack([B.r1(k) for k in range(N)])
        for bi in parts[si]:
            R2[blocks[bi]] = B.r2(*blocks[bi])
        if si == K - 1:
            ccsd_k.energy(P, t1 + R1 / D1, t2 + R2 / D2)
    dt = time.perf_counter() - t0
    v = 1.0 / dt
    cores = os.cpu_count()
    desc = ("the %d timed steps together form one complete oracle iteration of %s (block oracle, form A: "
            "F~ and R1 at every k, all %d R2 blocks, Jacobi update, energy) in %.1f s on the host cores"
            % (K, args.workload, len(blocks), dt))
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * dt / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "nk_grid": list(spec.grid), "nocc": spec.nocc, "nvir": spec.nvir,
                   "diis": WORKLOADS[args.workload]["diis_depth"]},
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_mixed(args, spec, dev, depth, local, fp64_solve, fp64_ms_per_iter):
    """The mixed form on the same inputs: iterations per second (traced) and the
    time to solution with FP64 polish, with |dE| against the FP64 solution."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Solver
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=1000,
               conv_tol=1e-12, mixed_tol=1e-7, polish_iters=2)
    for _ in range(args.warmup):
        S.iterate(1)
    torch.cuda.synchronize()
    S.trace(True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        S.iterate(1)
        launches += S.launches()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    steps = S.trace_steps()
    S.trace(False)
    S.close()
    tc = [s for s in steps if s[0] in ("ladder", "ring", "ring_W_t2", "hole_hole", "hole_hole_W")
          and s[3] > 0 and s[1] > 0 and s[3] / (s[2] / max(s[1], 1) / 1e3) > 20e12]   # tensor-core steps
    dom = max(tc, key=lambda s: s[2]) if tc else max(steps, key=lambda s: s[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / max(calls, 1) / 1e3
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops")
    peak = bf16 * TF32_NOMINAL_RATIO if bf16 else 1900.0 * TF32_NOMINAL_RATIO
    achieved = fl / avg_s / 1e12
    summ = {}
    for st in steps:
        if st[1]:
            summ[st[0]] = round(summ.get(st[0], 0.0) + st[2] / st[1], 3)
    out = {
        "value": 1e3 / ms, "unit": "iter/s", "ms_per_step": ms, "steps": args.steps, "gpu_launches": launches,
        "step_ms": summ,
        "precision": "tcgen05 split-TF32 (3 passes) for ladder, ring and hole-hole, FP32 CUDA cores elsewhere, FP64 update, DIIS and energy",
        "contraction_tflops": flops_per_iteration(spec) / (ms / 1e3) / 1e12,
        "speedup_per_iter_vs_fp64": fp64_ms_per_iter / ms,
        "roofline": {"kernel": f"tc_gemm_kernel ({name})", "bound": "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "executed_frac": 3.0 * achieved / peak,
                     "peak_source": ("measured bf16 %.0f TFLOP/s x nominal TF32/BF16 ratio" % bf16) if bf16
                     else "fallback 1.9 PFLOP/s bf16 x nominal TF32/BF16 ratio",
                     "flops_per_launch": fl, "launch_ms": avg_s * 1e3},
    }
    if fp64_solve is not None:
        S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=1000,
                   conv_tol=SOLVE_TOL, mixed_tol=1e-7, polish_iters=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok, iters, mr = S.solve()
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        e = S.energy().real
        S.close()
        # the same solve without the polish: the accuracy of the mixed iterations alone
        S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=1000,
                   conv_tol=SOLVE_TOL, mixed_tol=1e-7, polish_iters=0)
        S.solve()
        e0 = S.energy().real
        S.close()
        out["solve"] = {"converged_mixed_phase": ok, "iterations_incl_polish": iters, "polish_iters": 2,
                        "max_resid": mr, "seconds": secs, "e_per_cell": e,
                        "abs_dE_vs_fp64": abs(e - fp64_solve["e_per_cell"]),
                        "abs_dE_without_polish": abs(e0 - fp64_solve["e_per_cell"]),
                        "speedup_vs_fp64_solve": fp64_solve["seconds_est"] / secs}
        # the same solve with the polish iterations in the Ozaki form (FP64-accurate on the
        # BF16 tensor cores) instead of native FP64
        from paper_1911_00242_gb300.binding import CCSD_OZAKI
        S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=1000,
                   conv_tol=SOLVE_TOL, mixed_tol=1e-7, polish_iters=2, polish_precision=CCSD_OZAKI)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok2, iters2, mr2 = S.solve()
        torch.cuda.synchronize()
        secs2 = time.perf_counter() - t0
        e2 = S.energy().real
        S.close()
        out["solve_ozaki_polish"] = {"converged_mixed_phase": ok2, "iterations_incl_polish": iters2,
                                     "polish_iters": 2, "max_resid": mr2, "seconds": secs2, "e_per_cell": e2,
                                     "abs_dE_vs_fp64": abs(e2 - fp64_solve["e_per_cell"]),
                                     "speedup_vs_fp64_solve": fp64_solve["seconds_est"] / secs2}
    return out


def run_ozaki(args, spec, dev, depth, fp64_solve, fp64_ms_per_iter, slices=7):
    """The Ozaki form (FP64-accurate contractions on the BF16 tensor cores) on the same
    inputs: iterations per second (traced), roofline of its dominant tensor-core GEMM,
    and the time to solution with |dE| against the FP64 form's solution."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_OZAKI, Solver
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_OZAKI, diis_depth=depth, max_iter=1000,
               conv_tol=1e-12, oz_slices=slices)
    for _ in range(args.warmup):
        S.iterate(1)
    torch.cuda.synchronize()
    S.trace(True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        S.iterate(1)
        launches += S.launches()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    steps = S.trace_steps()
    S.trace(False)
    S.close()
    pairs = slices * (slices + 1) // 2
    tc = [s for s in steps if s[0] in ("ladder", "ring", "ring_W_t2", "hole_hole", "hole_hole_W")
          and s[3] > 0 and s[1] > 0 and s[3] / (s[2] / max(s[1], 1) / 1e3) > 5e12]   # tensor-core steps
    dom = max(tc, key=lambda s: s[2]) if tc else max(steps, key=lambda s: s[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / max(calls, 1) / 1e3
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops") or 1900.0
    achieved = fl / avg_s / 1e12
    summ = {}
    for st in steps:
        if st[1]:
            summ[st[0]] = round(summ.get(st[0], 0.0) + st[2] / st[1], 3)
    out = {
        "value": 1e3 / ms, "unit": "iter/s", "ms_per_step": ms, "steps": args.steps, "gpu_launches": launches,
        "step_ms": summ, "slices": slices,
        "precision": (f"Ozaki scheme: {slices} BF16 slices per operand row, {pairs} slice-pair products per "
                      "contraction on tcgen05 (exact FP32 windows, double-float sum) for ladder, ring, "
                      "hole-hole and F~_vv; double-float GEMMs elsewhere; FP64 update, DIIS and energy"),
        "contraction_tflops": flops_per_iteration(spec) / (ms / 1e3) / 1e12,
        "speedup_per_iter_vs_fp64": fp64_ms_per_iter / ms,
        "roofline": {"kernel": f"oz_gemm_kernel ({name})", "bound": "tensor", "achieved": achieved,
                     "peak": bf16, "unit": "TFLOP/s", "frac": achieved / bf16,
                     "executed_tflops": pairs * achieved, "executed_frac": pairs * achieved / bf16,
                     "peak_source": "measured bf16 %.0f TFLOP/s (of measured)" % bf16
                     if peaks.get("bf16_tflops") else "fallback 1.9 PFLOP/s bf16",
                     "flops_per_launch": fl, "launch_ms": avg_s * 1e3},
    }
    if fp64_solve is not None:
        S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_OZAKI, diis_depth=depth, max_iter=1000,
                   conv_tol=SOLVE_TOL, oz_slices=slices)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok, iters, mr = S.solve()
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        e = S.energy().real
        S.close()
        out["solve"] = {"converged": ok, "iterations": iters, "max_resid": mr, "seconds": secs, "e_per_cell": e,
                        "abs_dE_vs_fp64": abs(e - fp64_solve["e_per_cell"]),
                        "speedup_vs_fp64_solve": fp64_solve["seconds_est"] / secs}
    return out


def run_batch(args, local):
    """Batched form: 64 problems (N_k in {1,2,4,8}, o 4..8, v 8..24) per iteration."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_MIXED, BatchSolver
    specs = cs.batch_specs(64)
    if args.precision == "mixed":      # mixed members hold complex64 integrals
        specs = [cs.SynthSpec(**{**s.__dict__, "int_dtype": "c64"}) for s in specs]
    devs = [{k: torch.from_numpy(v).to(f"cuda:{local}") for k, v in cs.generate(s).items()} for s in specs]
    prec = CCSD_MIXED if args.precision == "mixed" else 0
    B = BatchSolver([(s.grid, s.nocc, s.nvir, d) for s, d in zip(specs, devs)], conv_tol=1e-30, precision=prec)
    t0 = time.perf_counter()
    B.iterate(1)                                 # autotune + graph capture + first iteration
    t_setup = time.perf_counter() - t0
    for _ in range(max(0, args.warmup - 1)):
        B.iterate(1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.iterate(1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    launches, cfgs = B.stats()
    fl = sum(flops_per_iteration(s) for s in specs)
    B.close()
    return {"metric": METRIC, "value": 64 * args.steps / dt, "unit": "member iter/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 integrals, mixed" if args.precision == "mixed" else "c128", "data": "synthetic",
            "config": {"workload": "batch64", "members": 64, "precision": args.precision,
                       "nk": [s.nk for s in specs], "nocc": [s.nocc for s in specs], "nvir": [s.nvir for s in specs]},
            "aggregate_tflops": fl * args.steps / dt / 1e12, "gpu_launches_per_step": launches,
            "gpu_launches": launches * args.steps, "clocks": clk,
            "timing": "host clock around the graph replays (each iteration ends with a copy of the member norms)",
            "autotune_and_capture_s": t_setup, "tile_cfgs": cfgs[:40]}


def run_serve(args, local):
    """Serving form: Poisson arrivals into the request loop; p50/p99 time to converge."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Server
    rng = np.random.default_rng([5000, 7])
    small = cs.batch_specs(16, seed=4000)
    large = cs.spec_for("grid222_o8_v32")
    pool = [(s, {k: torch.from_numpy(v).pin_memory() for k, v in cs.generate(s).items()}) for s in small]
    big = (large, {k: torch.from_numpy(v).pin_memory() for k, v in cs.generate(large).items()})
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=int(args.rate * args.duration * 2) + 10))
    arrivals = arrivals[arrivals < args.duration]
    picks = [(big if rng.random() < 0.1 else pool[int(rng.integers(0, len(pool)))]) for _ in arrivals]
    cfg = dict(conv_tol=1e-7, diis_depth=6, max_iter=200, precision=CCSD_MIXED, mixed_tol=1e-7, polish_iters=0)
    srv = Server(200 << 30, 32)
    clocks = ClockSampler(local)
    clocks.start()
    ids, t_start = [], time.perf_counter()
    peak_bytes = peak_active = 0
    for t_arr, (s, arr) in zip(arrivals, picks):
        while time.perf_counter() - t_start < t_arr:
            a, q, b = srv.stats()
            peak_bytes, peak_active = max(peak_bytes, b), max(peak_active, a)
            time.sleep(0.002)
        ids.append((srv.submit(s.grid, s.nocc, s.nvir, arr, **cfg), s is large))
    done = {}
    while len(done) < len(ids):
        for i, is_large in ids:
            if i not in done:
                st, e, t, it = srv.poll(i)
                if st == 2 or st < 0:
                    done[i] = (st, t, it, is_large)
        a, q, b = srv.stats()
        peak_bytes, peak_active = max(peak_bytes, b), max(peak_active, a)
        time.sleep(0.005)
    elapsed = time.perf_counter() - t_start
    clk = clocks.stop()
    prof = srv.profile()
    srv.close()
    ok = [v for v in done.values() if v[0] == 2]
    ts = np.array([v[1] for v in ok])
    tl = np.array([v[1] for v in ok if v[3]])
    tsm = np.array([v[1] for v in ok if not v[3]])
    q = lambda x, p: float(np.percentile(x, p)) if len(x) else None   # noqa: E731
    return {"metric": "CCSD solve time to converge", "value": q(ts, 99), "unit": "s (p99)", "n_gpus": 1,
            "steps": len(ids), "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed", "data": "synthetic",
            "config": {"workload": "serve", "rate_per_s": args.rate, "duration_s": args.duration,
                       "large_fraction": 0.1, "tolerance": 1e-7,
                       "policy": "tcgen05 split-TF32 mixed iterations to max|R| < 1e-7, DIIS(6), no FP64 polish",
                       "hbm_budget_gb": 200, "max_slots": 32},
            "p50_s": q(ts, 50), "p99_s": q(ts, 99), "p50_small_s": q(tsm, 50), "p99_small_s": q(tsm, 99),
            "p50_large_s": q(tl, 50), "p99_large_s": q(tl, 99),
            "solves_per_s": len(ok) / elapsed, "submitted": len(ids), "completed": len(ok),
            "failed": len(ids) - len(ok), "elapsed_s": elapsed, "peak_admitted_gb": peak_bytes / 2**30,
            "peak_active": peak_active, "clocks": clk,
            "server": prof}


def run_grid333(args, local):
    """Mixed-precision workload: 3x3x3 grid (N_k = 27), o 8, v 24, integrals stored
    complex64.  One step = one mixed iteration (tcgen05 split-TF32 contractions,
    FP64 update and DIIS(6)); the timed steps are the first iterations of a solve
    from t = 0 that continues to max|R| < 1e-7 and then runs 2 FP64 polish
    iterations.  The FP64 form on the same inputs (the same handle switched to
    FP64: the complex64 integrals widened exactly) is timed per iteration and
    continued from the polished amplitudes to max|R| < 1e-8 for the FP64 energy."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED, Solver
    spec = cs.spec_for("grid333_o8_v24_c64")
    device = f"cuda:{local}"
    t0 = time.perf_counter()
    dev = cs.generate_torch(spec, device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    if args.vvvv_on_host:       # vvvv stays in host memory, read in place by the kernels
        dev["vvvv"] = dev["vvvv"].cpu()
    torch.cuda.empty_cache()
    depth = WORKLOADS["grid333_o8_v24_c64"]["diis_depth"]
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=300,
               conv_tol=1e-8, mixed_tol=1e-7, polish_iters=2, vvvv_on_host=args.vvvv_on_host)
    free_b, total_b = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    t_solve0 = time.perf_counter()
    for _ in range(args.warmup):
        S.iterate(1)
    torch.cuda.synchronize()
    S.trace(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        S.iterate(1)
        launches += S.launches()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    steps = S.trace_steps()
    S.trace(False)
    ok, its, mr = S.solve()                  # the rest of the solve, then 2 FP64 polish iterations
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t_solve0
    mixed_iters = args.warmup + args.steps + its
    e_mixed = S.energy()

    # FP64 form on the same inputs: per-iteration time, then on to max|R| < 1e-8
    S.set_precision(CCSD_FP64)
    S.trace(True)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    fp64_timed = 2
    d = False
    for _ in range(fp64_timed):
        d, mr64 = S.iterate(1)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / fp64_timed
    fp64_steps = S.trace_steps()
    S.trace(False)
    extra = 0
    while not d and extra < 12:
        d, mr64 = S.iterate(1)
        extra += 1
    e_fp64 = S.energy()
    S.close()
    # the same solve without the polish: the accuracy of the mixed iterations alone
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=300,
               conv_tol=1e-8, mixed_tol=1e-7, polish_iters=0, vvvv_on_host=args.vvvv_on_host)
    t0 = time.perf_counter()
    S.solve()
    t_mixed_only = time.perf_counter() - t0
    e_mixed_only = S.energy()
    S.close()

    tc = [x for x in steps if x[3] > 0 and x[1] > 0 and x[3] / (x[2] / x[1] / 1e3) > 20e12]
    dom = max(tc, key=lambda x: x[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / calls / 1e3
    bf16 = measured_peaks().get("bf16_tflops")
    peak = (bf16 or 1900.0) * TF32_NOMINAL_RATIO
    achieved = fl / avg_s / 1e12
    summ = {}
    for x in steps:
        if x[1]:
            summ[x[0]] = round(summ.get(x[0], 0.0) + x[2] / x[1], 3)
    summ64 = {}
    for x in fp64_steps:
        if x[1]:
            summ64[x[0]] = round(summ64.get(x[0], 0.0) + x[2] / x[1], 1)
    fp64_solve_est = mixed_iters * fp64_ms / 1e3
    result = {
        "metric": METRIC, "value": 1e3 / ms, "unit": "iter/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed: tf32x3 contractions, fp64 update/DIIS/energy", "data": "synthetic",
        "config": {"workload": "grid333_o8_v24_c64", "nk_grid": list(spec.grid), "nocc": spec.nocc,
                   "nvir": spec.nvir, "int_dtype": "c64", "precision": "mixed", "diis": depth,
                   "parallelism": "single", "l2": "inputs larger than L2 (vvvv 52 GB)",
                   "input_synthesis_s": t_gen, "vvvv": "host memory, read in place" if args.vvvv_on_host
                   else "device memory", "device_gb_in_use": (total_b - free_b) / 1e9},
        "contraction_tflops": flops_per_iteration(spec) / (ms / 1e3) / 1e12,
        "roofline": {"kernel": f"tc_gemm_kernel ({name})", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "executed_frac": 3.0 * achieved / peak,
                     "peak_source": ("measured bf16 %.0f TFLOP/s x nominal TF32/BF16 ratio" % bf16) if bf16
                     else "fallback 1.9 PFLOP/s bf16 x nominal TF32/BF16 ratio",
                     "traffic": None, "flops_per_launch": fl, "launch_ms": avg_s * 1e3},
        "gpu_launches": launches, "clocks": clk, "step_ms": summ,
        "mixed_solve": {"converged": ok, "iterations_incl_polish": mixed_iters, "polish_iters": 2,
                        "max_resid": mr, "seconds": t_solve, "e_per_cell": e_mixed.real,
                        "e_imag": e_mixed.imag},
        "fp64": {"ms_per_iter": fp64_ms, "speedup_per_iter_mixed_vs_fp64": fp64_ms / ms,
                 "continued_iterations": fp64_timed + extra, "converged": bool(d), "max_resid": mr64,
                 "e_per_cell": e_fp64.real, "abs_dE_mixed_vs_fp64": abs(e_mixed.real - e_fp64.real),
                 "abs_dE_mixed_without_polish": abs(e_mixed_only.real - e_fp64.real),
                 "mixed_solve_without_polish_s": t_mixed_only,
                 "solve_seconds_est": fp64_solve_est,
                 "solve_est_basis": "FP64 from t = 0 taking the mixed solve's iteration count",
                 "speedup_solve_est": fp64_solve_est / t_solve, "step_ms": summ64},
    }
    del dev
    torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = grid333_cpu_baseline(spec)
    return result


def run_grid333_ozaki(args, local):
    """The 3x3x3/o8/v24 workload (complex64 integrals) in the Ozaki form: FP64-accurate
    contractions on the BF16 tensor cores, double-float elsewhere, FP64 update, DIIS and
    energy.  One step = one Ozaki iteration;
    the timed steps are the first iterations of a solve from t = 0 to max|R| < 1e-8.  The
    same handle then runs one native FP64 iteration from the converged amplitudes: its
    max|R| and energy change show how far the Ozaki fixed point is from the FP64 one.
    Last, the mixed form's solve with the Ozaki form as its polish (one handle carrying both
    tensor-core forms): mixed iterations to 1e-7, then Ozaki iterations to 1e-8."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED, CCSD_OZAKI, Solver
    spec = cs.spec_for("grid333_o8_v24_c64")
    device = f"cuda:{local}"
    t0 = time.perf_counter()
    dev = cs.generate_torch(spec, device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    torch.cuda.empty_cache()
    depth = WORKLOADS["grid333_o8_v24_c64"]["diis_depth"]
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_OZAKI, diis_depth=depth, max_iter=300,
               conv_tol=1e-8)
    free_b, total_b = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    t_solve0 = time.perf_counter()
    for _ in range(args.warmup):
        S.iterate(1)
    torch.cuda.synchronize()
    S.trace(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        S.iterate(1)
        launches += S.launches()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    steps = S.trace_steps()
    S.trace(False)
    ok, its, mr = S.solve()
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t_solve0
    iters = args.warmup + args.steps + its
    e_oz = S.energy()
    S.set_precision(CCSD_FP64)
    f0 = time.perf_counter()
    d, mr64 = S.iterate(1)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - f0
    e_fp64 = S.energy()
    S.close()
    del S
    # mixed iterations (tcgen05 split TF32) to max|R| < 1e-7, then polish iterations in the
    # Ozaki form instead of native FP64, to max|R| < 1e-8: one handle carrying both
    # tensor-core operand sets (they share the pooled buffers)
    m0 = time.perf_counter()
    M = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=300,
               conv_tol=1e-8, mixed_tol=1e-7, polish_iters=6, polish_precision=CCSD_OZAKI)
    t_create = time.perf_counter() - m0
    ok_mz, its_mz, mr_mz = M.solve()
    torch.cuda.synchronize()
    t_mz = time.perf_counter() - m0
    e_mz = M.energy()
    M.close()
    pairs = 28
    tc = [x for x in steps if x[3] > 0 and x[1] > 0 and x[0] in ("ladder", "ring", "ring_W_t2", "hole_hole",
                                                                   "hole_hole_W")]
    dom = max(tc, key=lambda x: x[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / calls / 1e3
    bf16 = measured_peaks().get("bf16_tflops") or 1900.0
    achieved = fl / avg_s / 1e12
    summ = {}
    for x in steps:
        if x[1]:
            summ[x[0]] = round(summ.get(x[0], 0.0) + x[2] / x[1], 3)
    return {
        "metric": METRIC, "value": 1e3 / ms, "unit": "iter/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "ozaki: 7 bf16 slices, exact fp32 windows, double-float sums; double-float and fp64 elsewhere",
        "data": "synthetic",
        "config": {"workload": "grid333_o8_v24_c64", "nk_grid": list(spec.grid), "nocc": spec.nocc,
                   "nvir": spec.nvir, "int_dtype": "c64", "precision": "ozaki", "diis": depth,
                   "parallelism": "single", "l2": "inputs larger than L2 (vvvv 52 GB)",
                   "input_synthesis_s": t_gen, "device_gb_in_use": (total_b - free_b) / 1e9},
        "contraction_tflops": flops_per_iteration(spec) / (ms / 1e3) / 1e12,
        "roofline": {"kernel": f"oz_gemm_kernel ({name})", "bound": "tensor", "achieved": achieved, "peak": bf16,
                     "unit": "TFLOP/s", "frac": achieved / bf16, "executed_frac": pairs * achieved / bf16,
                     "peak_source": "measured bf16 %.0f TFLOP/s (of measured)" % bf16, "traffic": None,
                     "flops_per_launch": fl, "launch_ms": avg_s * 1e3},
        "gpu_launches": launches, "clocks": clk, "step_ms": summ,
        "ozaki_solve": {"converged": ok, "iterations": iters, "max_resid": mr, "seconds": t_solve,
                        "e_per_cell": e_oz.real, "e_imag": e_oz.imag},
        "fp64_check": {"one_fp64_iteration_s": fp64_s, "fp64_max_resid_at_ozaki_solution": mr64,
                       "abs_dE_after_fp64_iteration": abs(e_fp64.real - e_oz.real)},
        "mixed_with_ozaki_polish": {"converged": ok_mz, "iterations_incl_polish": its_mz, "max_resid": mr_mz,
                                    "seconds_incl_create": t_mz, "create_s": t_create, "e_per_cell": e_mz.real,
                                    "abs_dE_vs_ozaki_solve": abs(e_mz.real - e_oz.real),
                                    "abs_dE_vs_fp64_iteration": abs(e_mz.real - e_fp64.real)},
    }


def grid333_block(args, local):
    """The mixed-precision workload inside the default line: 3x3x3 grid (N_k = 27), o 8,
    v 24, integrals stored complex64 (vvvv 52 GB), DIIS(6).  One handle carries the
    mixed form and its Ozaki polish.  Timed: `args.steps` mixed iterations (CUDA events,
    clocks sampled) after `args.warmup`; then the rest of the solve (mixed iterations to
    max|R| < 1e-7, Ozaki polish iterations to 1e-8); then the same handle switched to
    native FP64 runs one timed iteration from the polished amplitudes, whose max|R| and
    energy change give the distance to the FP64 fixed point."""
    import torch
    from paper_1911_00242_gb300.binding import CCSD_FP64, CCSD_MIXED, CCSD_OZAKI, Solver
    spec = cs.spec_for("grid333_o8_v24_c64")
    device = f"cuda:{local}"
    t0 = time.perf_counter()
    dev = cs.generate_torch(spec, device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    torch.cuda.empty_cache()
    depth = WORKLOADS["grid333_o8_v24_c64"]["diis_depth"]
    t_create0 = time.perf_counter()
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, precision=CCSD_MIXED, diis_depth=depth, max_iter=300,
               conv_tol=1e-8, mixed_tol=1e-7, polish_iters=6, polish_precision=CCSD_OZAKI)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t_create0
    free_b, total_b = torch.cuda.mem_get_info()
    stream = torch.cuda.current_stream()
    t_solve0 = time.perf_counter()
    for _ in range(args.warmup):
        S.iterate(1)
    torch.cuda.synchronize()
    S.trace(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        S.iterate(1)
        launches += S.launches()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    steps = S.trace_steps()
    S.trace(False)
    ok, its, mr = S.solve()                  # mixed iterations to 1e-7, then the Ozaki polish
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t_solve0
    iters = args.warmup + args.steps + its
    e_mixed = S.energy()
    S.set_precision(CCSD_FP64)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    d64, mr64 = S.iterate(1)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1)
    e_fp64 = S.energy()
    S.close()
    del S, dev
    torch.cuda.empty_cache()
    tc = [x for x in steps if x[3] > 0 and x[1] > 0 and x[3] / (x[2] / x[1] / 1e3) > 20e12]
    dom = max(tc, key=lambda x: x[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / calls / 1e3
    bf16 = measured_peaks().get("bf16_tflops")
    peak = (bf16 or 1900.0) * TF32_NOMINAL_RATIO
    achieved = fl / avg_s / 1e12
    return {
        "workload": "grid333_o8_v24_c64", "nk_grid": list(spec.grid), "nocc": spec.nocc, "nvir": spec.nvir,
        "int_dtype": "c64", "diis": depth, "input_synthesis_s": t_gen, "create_s": t_create,
        "device_gb_in_use": (total_b - free_b) / 1e9,
        "value": 1e3 / ms, "unit": "iter/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "gpu_launches": launches, "clocks": clk,
        "precision": "tcgen05 split-TF32 contractions, FP32 CUDA cores elsewhere, FP64 update/DIIS/energy",
        "contraction_tflops": flops_per_iteration(spec) / (ms / 1e3) / 1e12,
        "roofline": {"kernel": f"tc_gemm_kernel ({name})", "bound": "tensor", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "executed_frac": 3.0 * achieved / peak,
                     "peak_source": ("measured bf16 %.0f TFLOP/s x nominal TF32/BF16 ratio" % bf16) if bf16
                     else "fallback 1.9 PFLOP/s bf16 x nominal TF32/BF16 ratio",
                     "flops_per_launch": fl, "launch_ms": avg_s * 1e3},
        "solve": {"converged": ok, "iterations_incl_polish": iters, "polish": "Ozaki (FP64-accurate)",
                  "max_resid": mr, "seconds": t_solve, "e_per_cell": e_mixed.real},
        "fp64": {"ms_per_iter": fp64_ms, "speedup_per_iter_mixed_vs_fp64": fp64_ms / ms,
                 "max_resid_at_mixed_solution": mr64, "e_per_cell_after_fp64_iteration": e_fp64.real,
                 "abs_dE_mixed_vs_fp64_iteration": abs(e_mixed.real - e_fp64.real),
                 "solve_seconds_estimate": iters * fp64_ms / 1e3,
                 "solve_estimate_basis": "the mixed solve's iteration count at the measured FP64 time per iteration",
                 "speedup_solve_estimate": iters * fp64_ms / 1e3 / t_solve},
    }


def grid333_cpu_baseline(spec):
    """The block oracle on a bounded sample: the F~ intermediates (all k) and one R2
    block, scaled to a full iteration (N_k^3 blocks) -- the full oracle does not fit
    this workload."""
    from oracle.ccsd_k_block import BlockProblem, BlockResidual
    inp = {k: v.cpu().numpy() for k, v in cs.generate_torch(spec, "cuda").items()}
    import torch
    torch.cuda.empty_cache()
    t1, t2 = cs.random_amplitudes_torch(spec, 77, "cpu")
    B = BlockResidual(BlockProblem(spec.grid, spec.nocc, spec.nvir, inp), t1.numpy(), t2.numpy())
    t0 = time.perf_counter()
    B.fock()
    t_fock = time.perf_counter() - t0
    t0 = time.perf_counter()
    B.r2(1, 5, 26)
    t_blk = time.perf_counter() - t0
    secs = t_fock + t_blk * spec.nk ** 3
    return {"value": 1.0 / secs, "unit": "iter/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "block oracle: F~ at every k (%.1f s) plus one R2 block (%.1f s), scaled to the "
                      "N_k^3 = %d blocks of one iteration" % (t_fock, t_blk, spec.nk ** 3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="grid222_o8_v32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-form comparison")
    ap.add_argument("--no-ozaki", action="store_true", help="skip the Ozaki-form comparison")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-solution comparison")
    ap.add_argument("--no-grid333", action="store_true", help="skip the 3x3x3 mixed-precision block")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "ozaki"],
                    help="batch64: member precision (fp64, mixed); grid333_o8_v24_c64: ozaki runs that form")
    ap.add_argument("--rate", type=float, default=5.0, help="serve: requests per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--vvvv-on-host", action="store_true",
                    help="grid333_o8_v24_c64: keep vvvv in host memory (read in place over the host link)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    spec = cs.spec_for(args.workload) if args.workload in cs.CONFIGS else None

    if args.impl == "reference":
        if rank != 0:
            return 0
        if args.workload not in ("grid222_o8_v32", "grid221_o8_v32"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the FP64 "
                              "workloads (grid222_o8_v32, grid221_o8_v32)"}), flush=True)
            return 0
        print(json.dumps(run_reference(args, spec)), flush=True)
        return 0

    import torch
    torch.cuda.set_device(local)
    if args.workload == "batch64":
        print(json.dumps(run_batch(args, local)), flush=True)
        return 0
    if args.workload == "serve":
        print(json.dumps(run_serve(args, local)), flush=True)
        return 0
    if args.workload == "grid333_o8_v24_c64":
        run = run_grid333_ozaki if args.precision == "ozaki" else run_grid333
        print(json.dumps(run(args, local)), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1911_00242_gb300.binding import Solver

    peak64 = fp64_peak(local)
    inp = cs.generate(spec)
    dev = {k: torch.from_numpy(v).to(f"cuda:{local}") for k, v in inp.items()}
    depth = WORKLOADS[args.workload]["diis_depth"]
    S = Solver(spec.grid, spec.nocc, spec.nvir, dev, diis_depth=depth, max_iter=1000, conv_tol=SOLVE_TOL)
    zeros1 = torch.zeros((spec.nk, spec.nocc, spec.nvir), dtype=torch.complex128, device=f"cuda:{local}")
    zeros2 = torch.zeros((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, dtype=torch.complex128,
                         device=f"cuda:{local}")

    def step():
        done, mr = S.iterate(1)
        n = S.launches()
        if done:      # converged: restart from zero so that every step does a full iteration
            S.set_amplitudes(zeros1, zeros2)
        return n

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    S.trace(True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        launches += step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    steps = S.trace_steps()
    S.trace(False)
    energy = S.energy()
    ms = max_over_ranks(ms, dist, f"cuda:{local}")
    value = world * args.steps / (ms / 1e3)

    # dominant kernel: the plan step with the most device time
    dom = max(steps, key=lambda s: s[2])
    name, calls, tot_ms, fl, by = dom
    avg_s = tot_ms / max(calls, 1) / 1e3
    # The FP64 engine's algorithm is the 3M complex product: 3 FP64 FMAs (6 real flops) per
    # complex multiply-add, against the nominal 8 of the 4M count that the trace's flops use.
    # achieved and frac count the 3M flops against the FP64 rate measured on this GPU;
    # the nominal 4M rate is reported beside them.
    fl3 = 0.75 * fl
    achieved = fl3 / avg_s / 1e12
    pk = peak64["tflops"]
    roofline = {"kernel": f"zgemm_kb ({name})", "bound": "alu", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk,
                "flop_count": "3M: 6 real flops (3 FP64 FMAs) per complex multiply-add, the engine's algorithm",
                "nominal_4m_tflops": fl / avg_s / 1e12, "nominal_4m_frac": fl / avg_s / 1e12 / pk,
                "peak_source": ("measured in this run (ccsd_fp64_peak_probe, of measured): DFMA %.3f, FP64 mma.sync "
                                "%.3f TFLOP/s, SM clock median %s MHz while probing; the kernel ran at %s MHz"
                                % (peak64["dfma_tflops"], peak64["dmma_tflops"],
                                   (peak64["clocks"] or {}).get("sm_mhz"), (clk or {}).get("sm_mhz"))),
                "traffic": load_traffic(name), "flops_per_launch": fl3, "launch_ms": avg_s * 1e3}
    iter_flops = flops_per_iteration(spec)
    trace_summary = {}
    for st in steps:       # per step name: device ms per iteration, summed over its launches
        if st[1]:
            trace_summary[st[0]] = round(trace_summary.get(st[0], 0.0) + st[2] / st[1], 3)

    result = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "nk_grid": list(spec.grid), "nocc": spec.nocc, "nvir": spec.nvir,
                   "precision": "fp64", "diis": depth, "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (vvvv 8.6 GB)"},
        "contraction_tflops": iter_flops / (ms / args.steps / 1e3) / 1e12,
        "energy_per_cell": energy.real,
        "roofline": roofline,
        "gpu_launches": launches,
        "clocks": clk,
        "step_ms": trace_summary,
    }

    if not args.no_solve:
        # FP64 time to solution: continue the timed handle until max|R| < SOLVE_TOL
        # (the timed steps are the first iterations of this solve)
        t0 = time.perf_counter()
        ok, its, mres = S.solve()
        torch.cuda.synchronize()
        t_more = time.perf_counter() - t0
        fp64_iters = args.warmup + args.steps + its
        result["fp64_solve"] = {"converged": ok, "iterations": fp64_iters, "max_resid": mres,
                                "seconds_est": (args.warmup + args.steps) * ms / args.steps / 1e3 + t_more,
                                "e_per_cell": S.energy().real}

    if not args.no_mixed:
        result["mixed"] = run_mixed(args, spec, dev, depth, local, result.get("fp64_solve"), ms / args.steps)
    if not args.no_ozaki:
        result["ozaki"] = run_ozaki(args, spec, dev, depth, result.get("fp64_solve"), ms / args.steps)

    S.close()
    if not args.no_e2e:
        # end to end through the C ABI from pinned host buffers: create (copies
        # the integrals host->device), K iterations, energy, amplitudes back.
        host = {k: torch.from_numpy(v).pin_memory() for k, v in inp.items()}
        h1 = torch.empty(zeros1.shape, dtype=torch.complex128).pin_memory()
        h2 = torch.empty(zeros2.shape, dtype=torch.complex128).pin_memory()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        S2 = Solver(spec.grid, spec.nocc, spec.nvir, host, diis_depth=depth, max_iter=1000, conv_tol=1e-12)
        for _ in range(args.steps):
            S2.iterate(1)
        S2.energy()
        S2.get_amplitudes(h1, h2)
        S2.close()
        dt = time.perf_counter() - t0
        h2d = sum(v.nbytes for v in inp.values())
        d2h = h1.numel() * 16 + h2.numel() * 16
        result["e2e"] = {"value": world * args.steps / dt, "unit": "iter/s",
                         "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    if not args.no_grid333 and world == 1:
        # the mixed-precision workload (3x3x3, complex64 integrals) needs about 280 GB: the
        # FP64 workload's inputs are released first
        del dev, inp, zeros1, zeros2
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free_b, total_b = torch.cuda.mem_get_info()
        if total_b >= 250e9:
            result["grid333_mixed"] = grid333_block(args, local)
        else:
            result["grid333_mixed"] = {"skipped": "needs a GPU with about 280 GB of device memory"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, desc = cpu_oracle_iteration(args.workload)
        result["cpu_baseline"] = {"value": 1.0 / secs, "unit": "iter/s", "cores": os.cpu_count(), "kind": "oracle",
                                  "sample": desc}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
