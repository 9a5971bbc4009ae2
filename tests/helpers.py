"""Shared test helpers: dense (unfolded) views of a synthetic problem, and host builds
of the kernels' host-callable headers."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import ccsd_synth as cs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_host_probe(source, name):
    """Compiles tests/<source> (a host probe of a kernel header) into the repository's
    git-ignored _build/ folder and loads it; skips without nvcc.  -ffp-contract=off keeps
    every host floating-point operation a single rounding, as the device intrinsics are."""
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    nvcc = os.path.join(home, "bin", "nvcc")
    nvcc = nvcc if os.path.exists(nvcc) else shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    outdir = os.path.join(ROOT, "_build", "probes")
    os.makedirs(outdir, exist_ok=True)
    out = os.path.join(outdir, f"lib{name}_{os.getpid()}.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC,-ffp-contract=off", "-o", out, os.path.join(ROOT, "tests", source)],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    os.unlink(out)          # the loaded image stays mapped
    return lib


def dense_bloch(spec):
    """Dense Bloch-basis tensor and Fock built from the real-space supercell by an
    explicit unitary transform (independent of the generator's block DFT).
    Orbital order (k, p), p < o occupied."""
    V, f = cs.realspace_supercell(spec)
    nb = spec.nocc + spec.nvir
    U = cs.bloch_unitary(spec.grid, nb)
    Vk = np.einsum("ai,bj,ck,dl,abcd->ijkl", U.conj(), U.conj(), U, U, V, optimize=True)
    fk = U.conj().T @ f @ U
    N = spec.nk
    occ = [k * nb + i for k in range(N) for i in range(spec.nocc)]
    vir = [k * nb + spec.nocc + a for k in range(N) for a in range(spec.nvir)]
    return Vk, fk, occ, vir


def realspace(spec):
    V, f = cs.realspace_supercell(spec)
    nb = spec.nocc + spec.nvir
    N = spec.nk
    occ = [R * nb + i for R in range(N) for i in range(spec.nocc)]
    vir = [R * nb + spec.nocc + a for R in range(N) for a in range(spec.nvir)]
    return V, f, occ, vir


def k4(grid, a, b, c):
    n1, n2, n3 = grid
    def co(x):
        return np.array([x // (n2 * n3), (x // n3) % n2, x % n3])
    s = co(a) + co(b) - co(c)
    return int(((s[0] % n1) * n2 + (s[1] % n2)) * n3 + (s[2] % n3))


def to_dense(spec, t1, t2):
    """k-blocked amplitudes -> dense amplitudes over the (k, p) orbital order."""
    N, o, v = spec.nk, spec.nocc, spec.nvir
    T1 = np.zeros((N * o, N * v), complex)
    T2 = np.zeros((N * o, N * o, N * v, N * v), complex)
    for k in range(N):
        T1[k * o:(k + 1) * o, k * v:(k + 1) * v] = t1[k]
    for ki in range(N):
        for kj in range(N):
            for ka in range(N):
                kb = k4(spec.grid, ki, kj, ka)
                T2[ki * o:(ki + 1) * o, kj * o:(kj + 1) * o, ka * v:(ka + 1) * v, kb * v:(kb + 1) * v] = t2[ki, kj, ka]
    return T1, T2


def from_dense(spec, T1, T2):
    N, o, v = spec.nk, spec.nocc, spec.nvir
    t1 = np.stack([T1[k * o:(k + 1) * o, k * v:(k + 1) * v] for k in range(N)])
    t2 = np.zeros((N, N, N, o, o, v, v), complex)
    for ki in range(N):
        for kj in range(N):
            for ka in range(N):
                kb = k4(spec.grid, ki, kj, ka)
                t2[ki, kj, ka] = T2[ki * o:(ki + 1) * o, kj * o:(kj + 1) * o, ka * v:(ka + 1) * v, kb * v:(kb + 1) * v]
    return t1, t2
