"""Pins of the CPU oracle against what the paper and the mathematics fix.

1. MP2 closed form: with f_ov = 0, the first update t0 = f(0) (paper Sec. 3.2.2)
   is t2 = <ab||ij>/D, t1 = 0, so E(t0) = 1/4 sum |<ij||ab>|^2 / D.
2. Two-electron FCI: CCSD is exact for two electrons.
3. N_k = 1: the k-point code equals k-free molecular CCSD step by step.
4. Supercell unfolding: the k-point code equals molecular CCSD on the unfolded
   Bloch-basis tensor (step by step) and, at convergence, on the real-space
   localized basis (orbital-rotation invariance).
5. Form A (Sec. 2) = form B (Sec. 3.3) on random unconverged amplitudes.
6. Invariants: antisymmetry of R2, time reversal, coupling-constant scaling.
7. Convergence with and without DIIS to the same fixed point (Sec. 4.4), and the
   finite termination of DIIS on linear problems (its equivalence with GMRES).
"""
import numpy as np
import pytest

import ccsd_synth as cs
from helpers import dense_bloch, from_dense, realspace, to_dense
from oracle import ccsd_k, driver, fci, molecular
from oracle import ccsd_k_rearranged as form_b
from oracle.integrals import Integrals
from oracle.kmesh import KMesh


def problem(spec):
    return ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, cs.generate(spec))


def test_integral_access_all_classes():
    spec = cs.SynthSpec((2, 2, 1), 2, 3, 9, time_reversal=False)
    P = problem(spec)
    Vk, fk, occ, vir = dense_bloch(spec)
    N, o, v = spec.nk, spec.nocc, spec.nvir
    nb = o + v
    Vk = Vk.reshape(N, nb, N, nb, N, nb, N, nb)
    sl = {"o": slice(0, o), "v": slice(o, nb)}
    km = KMesh(spec.grid)
    for cls in (a + b + c + d for a in "ov" for b in "ov" for c in "ov" for d in "ov"):
        for kp in range(N):
            for kq in range(N):
                for kr in range(N):
                    ks = km.k4(kp, kq, kr)
                    ref = Vk[kp, sl[cls[0]], kq, sl[cls[1]], kr, sl[cls[2]], ks, sl[cls[3]]]
                    np.testing.assert_allclose(P.I.get(cls, kp, kq, kr), ref, atol=1e-15)


def test_kmesh():
    km = KMesh((2, 3, 4))
    for a in range(km.nk):
        assert km.add(a, km.neg(a)) == 0
        for b in range(km.nk):
            assert km.sub(km.add(a, b), b) == a
            assert km.k4(a, b, a) == b


def test_mp2_closed_form():
    spec = cs.SynthSpec((3, 1, 1), 2, 4, 13)
    P = problem(spec)
    r = driver.solve(P, n_iter=1)
    # closed form from the dense Bloch tensor, plain loops
    Vk, fk, occ, vir = dense_bloch(spec)
    e = 0.0
    for i in occ:
        for j in occ:
            for a in vir:
                for b in vir:
                    d = fk[i, i].real + fk[j, j].real - fk[a, a].real - fk[b, b].real
                    e += 0.25 * abs(Vk[i, j, a, b]) ** 2 / d
    assert abs(r["energies"][0] - e) < 1e-13
    assert np.all(r["t1"] == 0)


@pytest.mark.parametrize("grid,o,v,seed", [((1, 1, 1), 2, 4, 21), ((2, 1, 1), 1, 3, 22)])
def test_two_electron_fci(grid, o, v, seed):
    spec = cs.SynthSpec(grid, o, v, seed, time_reversal=False, fock_offdiag=0.1)
    P = problem(spec)
    r = driver.solve(P, tol=1e-12, max_iter=300)
    assert r["converged"]
    Vk, fk, occ, vir = dense_bloch(spec)
    e_fci = fci.correlation_energy(fk, Vk, occ)
    assert abs(r["energies"][-1] - e_fci) < 1e-10


def _compare_steps(spec, n_steps):
    P = problem(spec)
    Vk, fk, occ, vir = dense_bloch(spec)
    M = molecular.Dense(fk, Vk, occ, vir)
    t1, t2 = cs.random_amplitudes(spec, 5)
    T1, T2 = to_dense(spec, t1, t2)
    D1, D2 = driver.denominators(P)
    for _ in range(n_steps):
        R1, R2 = ccsd_k.residual(P, t1, t2)
        t1, t2 = t1 + R1 / D1, t2 + R2 / D2
        T1, T2 = molecular.step(M, T1, T2)
        k1, k2 = from_dense(spec, T1, T2)
        np.testing.assert_allclose(t1, k1, atol=1e-13)
        np.testing.assert_allclose(t2, k2, atol=1e-13)
        # the dense step keeps momentum conservation
        D1d, D2d = to_dense(spec, k1, k2)
        np.testing.assert_allclose(T2, D2d, atol=1e-13)
        assert abs(ccsd_k.energy(P, t1, t2) - molecular.energy(M, T1, T2)) < 1e-13


def test_nk1_equals_molecular():
    _compare_steps(cs.SynthSpec((1, 1, 1), 3, 4, 31, time_reversal=False, fock_offdiag=0.1), 3)


@pytest.mark.parametrize("tr", [True, False])
def test_unfolded_supercell_steps(tr):
    _compare_steps(cs.SynthSpec((2, 1, 1), 2, 3, 41, time_reversal=tr, fock_offdiag=0.05), 2)


def test_realspace_supercell_energy():
    spec = cs.SynthSpec((3, 1, 1), 1, 3, 51, time_reversal=False, fock_offdiag=0.05)
    P = problem(spec)
    r = driver.solve(P, tol=1e-11, max_iter=200)
    assert r["converged"]
    V, f, occ, vir = realspace(spec)
    e_rs, *_ = molecular.solve(molecular.Dense(f, V, occ, vir), tol=1e-12, max_iter=500)
    assert abs(r["energies"][-1] - e_rs) < 1e-9


@pytest.mark.parametrize("tr,off", [(True, 0.0), (False, 0.1)])
def test_form_a_equals_form_b(tr, off):
    spec = cs.SynthSpec((3, 1, 1), 2, 3, 61, time_reversal=tr, fock_offdiag=off)
    P = problem(spec)
    t1, t2 = cs.random_amplitudes(spec, 7)
    a1, a2 = ccsd_k.residual(P, t1, t2)
    b1, b2 = form_b.residual(P, t1, t2)
    np.testing.assert_allclose(b1, a1, atol=1e-14)
    np.testing.assert_allclose(b2, a2, atol=1e-14)


def test_form_a_equals_form_b_3d_grid():
    spec = cs.SynthSpec((2, 2, 1), 2, 2, 62, time_reversal=False, fock_offdiag=0.1)
    P = problem(spec)
    t1, t2 = cs.random_amplitudes(spec, 8)
    a1, a2 = ccsd_k.residual(P, t1, t2)
    b1, b2 = form_b.residual(P, t1, t2)
    np.testing.assert_allclose(b1, a1, atol=1e-14)
    np.testing.assert_allclose(b2, a2, atol=1e-14)


def test_residual_antisymmetry():
    spec = cs.SynthSpec((2, 2, 1), 2, 3, 71, time_reversal=False)
    P = problem(spec)
    t1, t2 = cs.random_amplitudes(spec, 9)
    _, R2 = ccsd_k.residual(P, t1, t2)
    km = P.km
    for ki in km:
        for kj in km:
            for ka in km:
                kb = km.k4(ki, kj, ka)
                np.testing.assert_allclose(R2[ki, kj, ka], -R2[kj, ki, ka].transpose(1, 0, 2, 3), atol=1e-15)
                np.testing.assert_allclose(R2[ki, kj, ka], -R2[ki, kj, kb].transpose(0, 1, 3, 2), atol=1e-15)


def test_time_reversal_invariants():
    spec = cs.SynthSpec((3, 1, 1), 2, 3, 81)
    P = problem(spec)
    r = driver.solve(P, tol=1e-10, max_iter=100)
    assert r["converged"]
    assert abs(r["energies"][-1].imag) < 1e-14
    km = P.km
    t1, t2 = r["t1"], r["t2"]
    for k in km:
        np.testing.assert_allclose(t1[km.neg(k)], np.conj(t1[k]), atol=1e-12)
    for ki in km:
        for kj in km:
            for ka in km:
                np.testing.assert_allclose(t2[km.neg(ki), km.neg(kj), km.neg(ka)], np.conj(t2[ki, kj, ka]),
                                           atol=1e-12)


def test_coupling_scaling():
    """E(lambda V) = lambda^2 E_MP2(V) + O(lambda^3)."""
    spec = cs.SynthSpec((2, 1, 1), 2, 3, 91)
    inp = cs.generate(spec)
    e_mp2 = driver.solve(ccsd_k.Problem(spec.grid, 2, 3, inp), n_iter=1)["energies"][0]
    errs = []
    for lam in (0.1, 0.05):
        x = dict(inp)
        for b in Integrals.STORED:
            x[b] = inp[b] * lam
        e = driver.solve(ccsd_k.Problem(spec.grid, 2, 3, x), tol=1e-14, max_iter=50)["energies"][-1]
        errs.append(abs(e - lam ** 2 * e_mp2))
    assert errs[0] < 1e-2 * abs(0.01 * e_mp2)
    assert 6.0 < errs[0] / errs[1] < 10.0   # third order


def test_chain_converges_with_and_without_diis():
    spec = cs.spec_for("chain_k4_o4_v8")
    P = problem(spec)
    a = driver.solve(P, tol=1e-8, max_iter=60)
    b = driver.solve(P, tol=1e-8, max_iter=60, diis_depth=6)
    assert a["converged"] and b["converged"]
    assert b["iters"] < a["iters"]
    assert abs(a["energies"][-1] - b["energies"][-1]) < 1e-8 * spec.nk


@pytest.mark.parametrize("spec", [cs.SynthSpec((2, 2, 1), 2, 3, 61, time_reversal=False, fock_offdiag=0.1),
                                  cs.SynthSpec((3, 1, 1), 2, 4, 62),
                                  cs.SynthSpec((2, 1, 1), 3, 2, 63, int_dtype="c64")],
                         ids=["complex", "real", "c64"])
def test_block_oracle_equals_full_oracle(spec):
    """ccsd_k_block (residual at chosen momentum blocks, for grids too large for the
    full oracle) reproduces ccsd_k.residual block by block; with complex64 inputs it
    widens each block exactly, as the full oracle does with widened arrays."""
    from oracle import ccsd_k_block
    inp = cs.generate(spec)
    t1, t2 = cs.random_amplitudes(spec, 3)
    P = ccsd_k.Problem(spec.grid, spec.nocc, spec.nvir, {k: np.asarray(v, np.complex128) for k, v in inp.items()})
    R1, R2 = ccsd_k.residual(P, t1, t2)
    B = ccsd_k_block.BlockResidual(ccsd_k_block.BlockProblem(spec.grid, spec.nocc, spec.nvir, inp), t1, t2)
    N = spec.nk
    for k in range(N):
        np.testing.assert_allclose(B.r1(k), R1[k], rtol=0, atol=1e-14)
    for ki in range(N):
        for kj in range(N):
            for ka in range(N):
                np.testing.assert_allclose(B.r2(ki, kj, ka), R2[ki, kj, ka], rtol=0, atol=1e-14)


def _linear_problem(rng, n, complex_=False):
    M = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if complex_ else 0)
    A = np.diag(rng.uniform(3, 5, n)) + 0.3 * (M + M.conj().T)
    b = rng.standard_normal(n) + (1j * rng.standard_normal(n) if complex_ else 0)
    return A, b, np.real(np.diag(A)).copy(), np.linalg.solve(A, b)


def _run_diis(diis, A, b, d, updates):
    """The driver's update (x + r/D, error r/D) on the linear problem A x = b."""
    x = np.zeros(len(b), np.result_type(A, b))
    for _ in range(updates):
        r = b - A @ x
        g = x + r / d
        x = diis.update(g, r / d) if diis is not None else g
    return x


def test_diis_terminates_on_linear_problems():
    """DIIS (Pulay extrapolation on the update errors, coefficients summing to one) is
    Anderson acceleration with full history, which on a linear fixed-point problem is
    equivalent to GMRES (Walker and Ni, SIAM J. Numer. Anal. 49 (2011) 1715): in exact
    arithmetic it reaches the solution of an n-dimensional real problem after n + 1
    updates, while the plain Jacobi step still converges linearly.  A Gram matrix of the
    amplitudes instead of the errors (a planted mistake) does not terminate."""
    rng = np.random.default_rng(31)
    for n in (3, 4, 6):
        A, b, d, xs = _linear_problem(rng, n)
        x = _run_diis(driver.DIIS(n + 2), A, b, d, n + 1)
        assert np.linalg.norm(x - xs) < 1e-12 * np.linalg.norm(xs)
        assert np.linalg.norm(_run_diis(None, A, b, d, n + 1) - xs) > 1e-6 * np.linalg.norm(xs)

        class GramOfAmplitudes(driver.DIIS):
            def update(self, x, e):
                return driver.DIIS.update(self, x, x)

        x = _run_diis(GramOfAmplitudes(n + 2), A, b, d, n + 1)
        assert np.linalg.norm(x - xs) > 1e-3 * np.linalg.norm(xs)
    # complex amplitudes: the real Gram matrix B_ij = Re <e_i|e_j> treats C^n as R^2n
    n = 4
    A, b, d, xs = _linear_problem(rng, n, complex_=True)
    x = _run_diis(driver.DIIS(2 * n + 2), A, b, d, 2 * n + 1)
    assert np.linalg.norm(x - xs) < 1e-12 * np.linalg.norm(xs)
