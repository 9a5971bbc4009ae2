"""The input generator: k-space blocks are the Bloch transform of the real-space
supercell Hamiltonian (paper Sec. 2, Sec. 3.2.5), with the symmetries of Sec. 3.3."""
import numpy as np
import pytest

import ccsd_synth as cs
from helpers import dense_bloch, k4


@pytest.mark.parametrize("tr", [True, False])
def test_blocks_are_bloch_transform_of_supercell(tr):
    spec = cs.SynthSpec((2, 2, 1), 2, 3, 7, time_reversal=tr, fock_offdiag=0.1)
    inp = cs.generate(spec)
    Vk, fk, occ, vir = dense_bloch(spec)
    N, o, v = spec.nk, spec.nocc, spec.nvir
    nb = o + v
    Vk = Vk.reshape(N, nb, N, nb, N, nb, N, nb)
    sl = {"o": slice(0, o), "v": slice(o, nb)}
    for b in cs.STORED_BLOCKS:
        for kp in range(N):
            for kq in range(N):
                for kr in range(N):
                    for ks in range(N):
                        ref = Vk[kp, sl[b[0]], kq, sl[b[1]], kr, sl[b[2]], ks, sl[b[3]]]
                        if ks == k4(spec.grid, kp, kq, kr):
                            np.testing.assert_allclose(inp[b][kp, kq, kr], ref, atol=1e-15)
                        else:   # momentum conservation
                            assert abs(ref).max() < 1e-15
    F = fk.reshape(N, nb, N, nb)
    for k in range(N):
        np.testing.assert_allclose(F[k, :o, k, :o], inp["f_oo"][k], atol=1e-14)
        np.testing.assert_allclose(F[k, o:, k, o:], inp["f_vv"][k], atol=1e-14)
        np.testing.assert_allclose(F[k, :o, k, o:], inp["f_ov"][k], atol=1e-14)


def test_block_symmetries_and_scale():
    spec = cs.SynthSpec((3, 1, 1), 2, 4, 3)
    inp = cs.generate(spec)
    N = spec.nk
    vv = inp["vvvv"]
    for kp in range(N):
        for kq in range(N):
            for kr in range(N):
                ks = k4(spec.grid, kp, kq, kr)
                b = vv[kp, kq, kr]
                np.testing.assert_allclose(b, -vv[kq, kp, kr].transpose(1, 0, 2, 3), atol=1e-16)
                np.testing.assert_allclose(b, -vv[kp, kq, ks].transpose(0, 1, 3, 2), atol=1e-16)
                np.testing.assert_allclose(b, np.conj(vv[kr, ks, kp].transpose(2, 3, 0, 1)), atol=1e-16)
                # time reversal of a real supercell tensor: V(-k) = V(k)^*
                m = [(-np.array([x])) % N for x in (kp, kq, kr)]
                np.testing.assert_allclose(vv[m[0][0], m[1][0], m[2][0]], np.conj(b), atol=1e-16)
    # std of the Bloch-normalized integrals is 0.05 / N (generic elements)
    big = cs.generate(cs.SynthSpec((2, 1, 1), 4, 12, 5), blocks=("vvvv",))["vvvv"]
    off = big[np.abs(big) > 0]
    assert 0.8 * 0.05 / 2 < np.sqrt(np.mean(np.abs(off) ** 2)) < 1.2 * 0.05 / 2


def test_seeded_and_layout():
    spec = cs.spec_for("chain_k4_o4_v8")
    a = cs.generate(spec, blocks=("oovv",))
    b = cs.generate(spec, blocks=("oovv",))
    assert np.array_equal(a["oovv"], b["oovv"])
    assert a["oovv"].shape == (4, 4, 4, 4, 4, 8, 8) and a["oovv"].flags.c_contiguous
    eo = np.real(np.einsum("kii->ki", a["f_oo"]))
    ev = np.real(np.einsum("kaa->ka", a["f_vv"]))
    assert eo.min() >= -1.5 and eo.max() <= -0.5 and ev.min() >= 0.5 and ev.max() <= 2.5
    assert np.all(a["f_ov"] == 0)


@pytest.mark.parametrize("spec", [cs.SynthSpec((2, 2, 1), 2, 3, 7, time_reversal=False, fock_offdiag=0.1),
                                  cs.SynthSpec((3, 1, 1), 2, 4, 3),
                                  cs.SynthSpec((2, 1, 1), 3, 2, 9, int_dtype="c64")],
                         ids=["complex", "real", "c64"])
def test_torch_evaluation_matches_generate(spec):
    """generate_torch() (the route for grids whose blocks do not fit the host twice) is
    the same recipe: the same draws, and values equal to generate() up to FFT rounding
    (complex128), or to one rounding to complex64."""
    torch = pytest.importorskip("torch")
    a = cs.generate(spec)
    b = cs.generate_torch(spec, "cpu")
    for k in a:
        y = b[k].numpy()
        assert y.dtype == a[k].dtype and y.shape == a[k].shape
        tol = 1e-15 if a[k].dtype == np.complex128 else 2e-9
        assert np.abs(a[k] - y).max() <= tol, k
    t1a, t2a = cs.random_amplitudes_slabs(spec, 5)
    t1b, t2b = cs.random_amplitudes_torch(spec, 5, "cpu")
    assert np.array_equal(t1a, t1b.numpy()) and np.array_equal(t2a, t2b.numpy())


def test_slab_amplitudes_antisymmetric_and_conserving():
    spec = cs.SynthSpec((3, 2, 1), 2, 3, 13)
    t1, t2 = cs.random_amplitudes_slabs(spec, 8)
    N = spec.nk
    for ki in range(N):
        for kj in range(N):
            for ka in range(N):
                kb = k4(spec.grid, ki, kj, ka)
                b = t2[ki, kj, ka]
                np.testing.assert_allclose(b, -t2[kj, ki, ka].transpose(1, 0, 2, 3), rtol=0, atol=1e-16)
                np.testing.assert_allclose(b, -t2[ki, kj, kb].transpose(0, 1, 3, 2), rtol=0, atol=1e-16)
    assert np.abs(t2).max() > 0 and np.abs(t1).max() > 0
