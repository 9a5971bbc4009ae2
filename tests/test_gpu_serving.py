"""Serving form: continuous batching of solves in a request loop.

Each solve must give the same result alone and in the mix (it runs the same
kernels on the same data; concurrency only interleaves independent streams),
admission must respect the memory budget, and oversized requests fail cleanly."""
import time

import numpy as np
import pytest

import ccsd_synth as cs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [
    cs.SynthSpec((2, 1, 1), 3, 5, 3001),
    cs.SynthSpec((1, 1, 1), 4, 8, 3002, time_reversal=False),
    cs.SynthSpec((2, 2, 1), 2, 4, 3003),
    cs.SynthSpec((4, 1, 1), 4, 6, 3004),
    cs.SynthSpec((2, 1, 1), 5, 9, 3005),
]


def wait_all(srv, ids, timeout=300.0):
    t0 = time.time()
    out = {}
    while len(out) < len(ids):
        for i in ids:
            if i in out:
                continue
            st, e, t, it = srv.poll(i)
            if st == 2 or st < 0:
                out[i] = (st, e, t, it)
        assert time.time() - t0 < timeout, "serving loop did not finish"
        time.sleep(0.01)
    return out


def standalone(spec, inp, **cfg):
    from paper_1911_00242_gb300.binding import Solver
    S = Solver(spec.grid, spec.nocc, spec.nvir, inp, **cfg)
    ok, it, mr = S.solve()
    e = S.energy().real
    S.close()
    return ok, e


@pytest.mark.parametrize("precision", [0, 1])
def test_results_alone_equal_results_in_mix(lib, precision):
    from paper_1911_00242_gb300.binding import Server
    cfg = dict(conv_tol=1e-8, diis_depth=6, max_iter=100, precision=precision, mixed_tol=1e-7, polish_iters=2)
    inps = [cs.generate(s) for s in SPECS]
    srv = Server(64 << 30, 8)
    ids = [srv.submit(s.grid, s.nocc, s.nvir, inp, **cfg) for s, inp in zip(SPECS, inps)]
    res = wait_all(srv, ids)
    srv.close()
    for s, inp, i in zip(SPECS, inps, ids):
        st, e, t, it = res[i]
        assert st == 2, (s, st)
        ok, e_alone = standalone(s, inp, **cfg)
        assert e == e_alone, (s, e, e_alone)
        assert t > 0 and it > 0


def test_admission_by_footprint(lib):
    from paper_1911_00242_gb300 import binding
    from paper_1911_00242_gb300.binding import Server
    import ctypes
    inps = [cs.generate(s) for s in SPECS]
    fp = []
    for s in SPECS:
        c = binding.make_config(s.grid, s.nocc, s.nvir)
        n = ctypes.c_size_t(0)
        assert lib.ccsd_footprint(ctypes.byref(c), 0, binding.CCSD_C128, ctypes.byref(n)) == 0
        fp.append(n.value)
    budget = max(fp) + min(fp)                 # at most two at a time
    srv = Server(budget, 8)
    ids = [srv.submit(s.grid, s.nocc, s.nvir, inp, conv_tol=1e-8, max_iter=100) for s, inp in zip(SPECS, inps)]
    peak_queued, peak_bytes = 0, 0
    done = {}
    t0 = time.time()
    while len(done) < len(ids):
        a, q, b = srv.stats()
        peak_queued = max(peak_queued, q)
        peak_bytes = max(peak_bytes, b)
        assert b <= budget
        for i in ids:
            if i not in done:
                st, e, t, it = srv.poll(i)
                if st == 2 or st < 0:
                    done[i] = st
        assert time.time() - t0 < 300
        time.sleep(0.005)
    srv.close()
    assert all(st == 2 for st in done.values())
    assert peak_queued > 0
    # a request larger than the whole budget fails with CCSD_ERR_OOM instead of waiting forever
    srv = Server(min(fp) // 2, 2)
    i = srv.submit(SPECS[0].grid, SPECS[0].nocc, SPECS[0].nvir, inps[0])
    st = wait_all(srv, [i])[i][0]
    srv.close()
    assert st == -2


def test_served_energies_match_oracle(lib):
    """Served solves against the oracle (paper Sec. 4.4 iteration, DIIS(6)): two FP64
    solves and one mixed solve with its FP64 polish, converged to max|R| < 1e-7 (the
    serving tolerance) in one mix on a caller-given stream; each energy per cell is
    within 1e-7 Ha of the oracle's energy converged to 1e-10."""
    from oracle import ccsd_k, driver
    from paper_1911_00242_gb300.binding import CCSD_MIXED, Server
    reqs = [(SPECS[0], 0), (SPECS[2], 0), (SPECS[3], CCSD_MIXED)]
    inps = [cs.generate(s) for s, _ in reqs]
    stream = torch.cuda.Stream()
    srv = Server(64 << 30, 8, stream=stream.cuda_stream)
    ids = [srv.submit(s.grid, s.nocc, s.nvir, inp, conv_tol=1e-7, diis_depth=6, max_iter=100, precision=p,
                      mixed_tol=1e-7, polish_iters=2)
           for (s, p), inp in zip(reqs, inps)]
    res = wait_all(srv, ids)
    srv.close()
    for (s, p), inp, i in zip(reqs, inps, ids):
        st, e, t, it = res[i]
        assert st == 2, (s, st)
        P = ccsd_k.Problem(s.grid, s.nocc, s.nvir, inp)
        ref = driver.solve(P, tol=1e-10, max_iter=200, diis_depth=6)
        assert ref["converged"]
        de = abs(e - ref["energies"][-1].real / s.nk)
        print(f"served {s.grid} o{s.nocc} v{s.nvir} precision {p}: |dE| vs oracle {de:.1e}")
        assert de < 1e-7, (s, p, e, de)


def test_sequential_requests_rebuild_their_groups(lib):
    """One slot: each request is admitted only after the previous one retired, so a new
    request can get the address of a retired handle.  Its round groups must be built
    for it (they are keyed by request id), and every result equals the solve alone."""
    from paper_1911_00242_gb300.binding import Server
    specs = [cs.SynthSpec((2, 1, 1), o, v, 3100 + i) for i, (o, v) in enumerate([(3, 5), (2, 4), (4, 6), (3, 7)])]
    inps = [cs.generate(s) for s in specs]
    cfg = dict(conv_tol=1e-8, diis_depth=6, max_iter=100)
    srv = Server(64 << 30, 1)
    ids = [srv.submit(s.grid, s.nocc, s.nvir, inp, **cfg) for s, inp in zip(specs, inps)]
    res = wait_all(srv, ids)
    srv.close()
    for s, inp, i in zip(specs, inps, ids):
        st, e, t, it = res[i]
        assert st == 2, (s, st)
        ok, e_alone = standalone(s, inp, **cfg)
        assert e == e_alone, (s, e, e_alone)
