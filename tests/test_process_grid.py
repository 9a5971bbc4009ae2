"""The paper's N_k^2 process-grid schedule (Sec. 3.2 data placement, Table 1,
the communication procedures of Sec. 4.3, the steps of Sec. 4.4), emulated on
host ranks, against the oracle: the distributed right-hand sides equal form A
block by block, iterations equal the oracle's Jacobi iterations, and the same
program runs as separate gloo processes."""
import os
import socket
import tempfile

import numpy as np
import pytest

import ccsd_synth as cs
from oracle import ccsd_k, driver, process_grid as pg

GRIDS = [cs.SynthSpec((2, 1, 1), 2, 3, 5, time_reversal=False, fock_offdiag=0.05),
         cs.SynthSpec((3, 1, 1), 2, 3, 6),
         cs.SynthSpec((2, 2, 1), 2, 3, 7, time_reversal=False)]


@pytest.mark.parametrize("spec", GRIDS, ids=lambda s: f"{s.grid}")
def test_distributed_residual_equals_oracle(spec):
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 4)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    G1, G2, stats = pg.run_threads(spec.grid, spec.nocc, spec.nvir, inp, t1, t2)
    np.testing.assert_allclose(G1, R1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(G2, R2, rtol=0, atol=1e-14)
    # every procedure of Sec. 4.3 moved data
    for name in ("reduce_horizontal", "reduce_vertical", "bcast_vertical", "allgather_horizontal",
                 "alltoall_horizontal", "alltoall_vertical", "sum88_shift", "diag_swap"):
        assert stats[name][0] > 0, name


def test_distributed_iterations_equal_oracle():
    """Jacobi iterations from t = 0 (t0 = f(0), Sec. 3.2.2), with the global max|R|
    test, on the 1D chain grid: the same iterates and norms as the oracle's driver."""
    spec = cs.SynthSpec((4, 1, 1), 2, 4, 8)
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    norms = []
    ref = driver.solve(P, n_iter=3, callback=lambda it, a, b, e: None)
    z1 = np.zeros((spec.nk, spec.nocc, spec.nvir), np.complex128)
    z2 = np.zeros((spec.nk,) * 3 + (spec.nocc,) * 2 + (spec.nvir,) * 2, np.complex128)
    T1, T2, norms, stats = pg.run_threads(spec.grid, spec.nocc, spec.nvir, inp, z1, z2, n_iter=3)
    np.testing.assert_allclose(T1, ref["t1"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(T2, ref["t2"], rtol=0, atol=1e-13)
    assert len(norms) == 3 and norms[0] > norms[1] > norms[2]


def test_table1_locality_is_enforced(monkeypatch):
    """A placement that contradicts the schedule is caught: with vvvv held by
    (kb, ka) instead of (ka, kb) the A-check step reads a block its rank does not hold."""
    spec = GRIDS[0]
    inp = cs.generate(spec)
    t1, t2 = cs.random_amplitudes(spec, 4)
    monkeypatch.setitem(pg.TABLE1, "vvvv", (lambda a, b, c, d: (b, a) if a != b else (a, (a + 1) % 2),))
    with pytest.raises(pg.LocalityError):
        pg.run_threads(spec.grid, spec.nocc, spec.nvir, inp, t1, t2)


def _gloo_rank(rank, world, port, path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    spec = GRIDS[0]
    N = spec.nk
    inp = cs.generate(spec)
    t1, t2 = cs.random_amplitudes(spec, 4)
    comm = pg.GlooComm(N, dist)
    alpha, beta = rank % N, rank // N
    rk = pg.Rank(alpha, beta, spec.grid, spec.nocc, spec.nvir, inp, comm)
    r1, s2 = pg.residual_program(rk, t1, pg.local_t2(t2, alpha, beta, N))
    got = comm.gather_all(rk, (r1, s2, comm.stats))
    if rank == 0:
        np.save(path, np.array([got], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_processes_run_the_same_schedule():
    """One gloo process per rank (N_k = 2: four processes) produces the oracle's
    residual and moves the same bytes per procedure as the thread transport."""
    import torch.multiprocessing as mp
    spec = GRIDS[0]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "gloo.npy")
        mp.start_processes(_gloo_rank, args=(spec.nk ** 2, port, path), nprocs=spec.nk ** 2, start_method="spawn")
        got = np.load(path, allow_pickle=True)[0]
    inp = cs.generate(spec)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, inp)
    t1, t2 = cs.random_amplitudes(spec, 4)
    R1, R2 = ccsd_k.residual(P, t1, t2)
    G1 = np.zeros_like(R1)
    G2 = np.zeros_like(R2)
    gloo_bytes = {}
    for r, (r1, s2, st) in got.items():
        if r1 is not None:
            G1[r % spec.nk] = r1
        for (ki, kj, ka), blk in s2.items():
            G2[ki, kj, ka] = blk
        for k, (b, m) in st.items():
            gloo_bytes[k] = gloo_bytes.get(k, 0) + b
    np.testing.assert_allclose(G1, R1, rtol=0, atol=1e-14)
    np.testing.assert_allclose(G2, R2, rtol=0, atol=1e-14)
    _, _, stats = pg.run_threads(spec.grid, spec.nocc, spec.nvir, inp, t1, t2)
    for k, (b, m) in stats.items():
        assert gloo_bytes[k] == b, k
