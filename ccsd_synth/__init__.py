"""Seeded synthetic inputs for periodic spin-orbital CCSD.

This module only produces inputs: Fock blocks and antisymmetrized two-electron
integral blocks of a translation-invariant supercell Hamiltonian, in the block
layout shared by the CPU oracle and the GPU library.  It contains none of the
CCSD arithmetic.

Physical model
--------------
A Born-von Karman supercell of N = n1*n2*n3 cells carries nb = o + v spin
orbitals chi_{p,R} per cell (the first o are occupied, the rest virtual).
A raw real tensor G[p R1, q R2, r R3, s 0] (the fourth cell pinned at the
origin, translation invariance gives every other element) is drawn from
N(0, 1), one independent stream per orbital-class tuple and per first
orbital.  It is antisymmetrized,
    A = G - G(p<->q) - G(r<->s) + G(p<->q, r<->s),
Hermitized, H = (A + A^dagger) / 2, and scaled so that a generic element of
the per-cell Fourier sum N <pq||rs> (the integral before the 1/N of the Bloch
normalization) has standard deviation 0.05 Ha; the integrals themselves then
have standard deviation 0.05 / N, which keeps per-cell energies intensive.

Bloch orbitals phi_{p k} = N^{-1/2} sum_R exp(i k.R) chi_{p R} turn it into
k-conserving blocks (paper Sec. 2 and Sec. 3.2.5):
    <p kp q kq || r kr s ks> = N^{-1} sum_{R1,R2,R3} exp(-i kp.R1 - i kq.R2 + i kr.R3)
                               H[p R1, q R2, r R3, s 0]
whenever kp + kq = kr + ks on the grid, and 0 otherwise.

Layouts (row-major, last index fastest, complex interleaved re/im)
------------------------------------------------------------------
    f_oo[k][i][j], f_vv[k][a][b], f_ov[k][i][a]
    B[kp][kq][kr][p][q][r][s]  for B in oooo, ooov, oovv, ovvo, ovvv, vvvv
      (ks implied by kp + kq - kr, componentwise modulo the grid)
    t1[k][i][a], t2[ki][kj][ka][i][j][a][b] (kb implied)
A k point is the integer triple (k1, k2, k3), 0 <= kd < nd, flattened as
(k1 * n2 + k2) * n3 + k3; cells R use the same flattening.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

__all__ = [
    "SynthSpec", "CONFIGS", "spec_for", "batch_specs", "generate", "generate_fock",
    "realspace_supercell", "bloch_unitary", "STORED_BLOCKS", "random_amplitudes",
    "generate_torch", "random_amplitudes_slabs", "random_amplitudes_torch",
]

STORED_BLOCKS = ("oooo", "ooov", "oovv", "ovvo", "ovvv", "vvvv")
K_STD = 0.05


@dataclass(frozen=True)
class SynthSpec:
    grid: tuple          # (n1, n2, n3)
    nocc: int            # occupied spin orbitals per k
    nvir: int            # virtual spin orbitals per k
    seed: int
    time_reversal: bool = True   # real real-space tensor and eps(k) = eps(-k)
    fock_offdiag: float = 0.0    # magnitude of random off-diagonal Fock (incl. f_ov)
    int_dtype: str = "c128"      # "c128" or "c64" for the integral blocks

    @property
    def nk(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]


# The workloads: a 1D chain (parity), the FP64 3D grid, the mixed-precision
# 3D grid.  Seeds are 1000 + workload number.
CONFIGS = {
    "chain_k4_o4_v8": SynthSpec((4, 1, 1), 4, 8, 1001),
    "grid222_o8_v32": SynthSpec((2, 2, 2), 8, 32, 1002),
    "grid333_o8_v24_c64": SynthSpec((3, 3, 3), 8, 24, 1003, int_dtype="c64"),
    # smaller grid with the FP64 workload's orbitals, for profiling captures
    "grid221_o8_v32": SynthSpec((2, 2, 1), 8, 32, 1012),
}


BATCH_GRIDS = ((1, 1, 1), (2, 1, 1), (2, 2, 1), (2, 2, 2))      # N_k in {1, 2, 4, 8}


def batch_specs(count: int = 64, seed: int = 2000) -> list:
    """The batched workload: `count` independent problems, N_k drawn from
    {1, 2, 4, 8}, n_occ uniform in 4..8, n_vir uniform in 8..24 (one size
    stream seeded with `seed`), instance i seeded seed + i."""
    rng = np.random.default_rng([seed, 41])
    out = []
    for i in range(count):
        g = BATCH_GRIDS[int(rng.integers(0, len(BATCH_GRIDS)))]
        o = int(rng.integers(4, 9))
        v = int(rng.integers(8, 25))
        out.append(SynthSpec(g, o, v, seed + i))
    return out


def spec_for(name: str, **over) -> SynthSpec:
    s = CONFIGS[name]
    if over:
        d = dict(s.__dict__)
        d.update(over)
        s = SynthSpec(**d)
    return s


# ----------------------------------------------------------------- k grid
def _coords(grid):
    n1, n2, n3 = grid
    idx = np.arange(n1 * n2 * n3)
    return np.stack([idx // (n2 * n3), (idx // n3) % n2, idx % n3], axis=1)


def _flat(grid, c):
    n1, n2, n3 = grid
    c = np.asarray(c)
    return ((c[..., 0] % n1) * n2 + (c[..., 1] % n2)) * n3 + (c[..., 2] % n3)


def _ks_table(grid):
    """ks[kp, kq, kr] = kp + kq - kr on the grid (the input layout's implied index)."""
    c = _coords(grid)
    s = c[:, None, None, :] + c[None, :, None, :] - c[None, None, :, :]
    return _flat(grid, s)


def _neg(grid):
    return _flat(grid, -_coords(grid))


def _cell_diff(grid):
    """d[R, R'] = R - R' on the cell grid."""
    c = _coords(grid)
    return _flat(grid, c[:, None, :] - c[None, :, :])


def _phase(grid):
    """phi[k, R] = exp(-i k.R), k.R = 2 pi sum_d k_d R_d / n_d."""
    c = _coords(grid).astype(np.float64)
    n = np.asarray(grid, dtype=np.float64)
    kr = (c[:, None, :] * c[None, :, :] / n).sum(-1)
    return np.exp(-2j * np.pi * kr)


# ------------------------------------------------------------ random draws
def _class_code(cls: str) -> int:
    return sum((1 << (3 - i)) for i, c in enumerate(cls) if c == "v")


def _draw_slice(spec: SynthSpec, cls: str, p: int) -> np.ndarray:
    """Raw tensor slice G_cls[p, R1, q, R2, r, R3, s] for one first orbital p.

    Shape (N, n_q, N, n_r, N, n_s).  One independent stream per (class, p)."""
    n = {"o": spec.nocc, "v": spec.nvir}
    N = spec.nk
    shape = (N, n[cls[1]], N, n[cls[2]], N, n[cls[3]])
    rng = np.random.default_rng([spec.seed, 17, _class_code(cls), p])
    g = rng.standard_normal(shape)
    if not spec.time_reversal:
        g = (g + 1j * rng.standard_normal(shape)) * (1.0 / math.sqrt(2.0))
    return g


def _scale(spec: SynthSpec) -> float:
    # A generic element of the Fourier sum N <pq||rs> of the raw tensor has
    # E|.|^2 = 2 N^3 (N^3 cell triples, four raw terms, then the Hermitian
    # average of two independent ones).  K_STD is the standard deviation of
    # that per-cell sum, so the Bloch-normalized integrals have std K_STD / N.
    N = spec.nk
    return K_STD / math.sqrt(2.0 * N ** 3)


def _gk(spec: SynthSpec, cls: str) -> np.ndarray:
    """Bloch transform of the raw class tensor: (N, N, N, n_p, n_q, n_r, n_s).

    The three cell sums are 3D discrete Fourier transforms on the grid:
    exp(-i k.R) for R1 and R2 (forward FFT), exp(+i k.R) for R3 (unnormalized
    inverse FFT), times 1/N."""
    n = {"o": spec.nocc, "v": spec.nvir}
    N = spec.nk
    g3 = tuple(spec.grid)
    out = np.empty((N, N, N, n[cls[0]], n[cls[1]], n[cls[2]], n[cls[3]]), np.complex128)

    def one(p):
        g = _draw_slice(spec, cls, p)                        # (R1, q, R2, r, R3, s)
        nq, nr, ns = g.shape[1], g.shape[3], g.shape[5]
        x = g.reshape(g3 + (nq,) + g3 + (nr,) + g3 + (ns,))
        x = sfft.fftn(x, axes=(0, 1, 2, 4, 5, 6), workers=1)
        x = sfft.ifftn(x, axes=(8, 9, 10), norm="forward", workers=1, overwrite_x=True)
        x = x.reshape(N, nq, N, nr, N, ns)
        out[:, :, :, p] = x.transpose(0, 2, 4, 1, 3, 5)

    _pmap(one, range(n[cls[0]]))
    out *= 1.0 / N
    return out


def _pmap(fn, items):
    items = list(items)
    workers = min(len(items), os.cpu_count() or 1, 16)
    if workers <= 1:
        for x in items:
            fn(x)
        return
    with ThreadPoolExecutor(workers) as ex:
        for _ in ex.map(fn, items):
            pass


def _swap(cls, perm):
    return "".join(cls[i] for i in perm)


def _antisym(spec, cls, gk_cache, ks):
    """A_cls[kp,kq,kr] = G - G(bra swap) - G(ket swap) + G(both), in k space."""
    N = spec.nk
    def g(c):
        if c not in gk_cache:
            gk_cache[c] = _gk(spec, c)
        return gk_cache[c]
    g0 = g(cls)
    gb = g(_swap(cls, (1, 0, 2, 3)))
    gk_ = g(_swap(cls, (0, 1, 3, 2)))
    gbk = g(_swap(cls, (1, 0, 3, 2)))
    A = np.empty_like(g0)

    def one(kp):
        for kq in range(N):
            for kr in range(N):
                kz = ks[kp, kq, kr]
                a = g0[kp, kq, kr] - gb[kq, kp, kr].transpose(1, 0, 2, 3)
                a -= gk_[kp, kq, kz].transpose(0, 1, 3, 2)
                a += gbk[kq, kp, kz].transpose(1, 0, 3, 2)
                A[kp, kq, kr] = a

    _pmap(one, range(N))
    return A


def _block(spec: SynthSpec, cls: str, ks) -> np.ndarray:
    cache = {}
    A = _antisym(spec, cls, cache, ks)
    hc = _swap(cls, (2, 3, 0, 1))
    Ah = A if hc == cls else _antisym(spec, hc, cache, ks)
    cache.clear()
    N = spec.nk
    H = np.empty_like(A)
    sc = 0.5 * _scale(spec)

    def one(kp):
        for kq in range(N):
            for kr in range(N):
                kz = ks[kp, kq, kr]
                # conj(A_h[kr, ks, kp](r, s, p, q)) arranged as [p, q, r, s]
                h = A[kp, kq, kr] + np.conj(Ah[kr, kz, kp]).transpose(2, 3, 0, 1)
                h *= sc
                H[kp, kq, kr] = h

    _pmap(one, range(N))
    del A, Ah
    return H


def generate_fock(spec: SynthSpec):
    """f_oo (N,o,o), f_vv (N,v,v), f_ov (N,o,v), complex128, Hermitian per k."""
    N, o, v = spec.nk, spec.nocc, spec.nvir
    rng = np.random.default_rng([spec.seed, 23])
    eo = rng.uniform(-1.5, -0.5, (N, o))
    ev = rng.uniform(0.5, 2.5, (N, v))
    neg = _neg(spec.grid)
    if spec.time_reversal:
        for k in range(N):
            if neg[k] < k:
                eo[k], ev[k] = eo[neg[k]], ev[neg[k]]
    f_oo = np.zeros((N, o, o), np.complex128)
    f_vv = np.zeros((N, v, v), np.complex128)
    f_ov = np.zeros((N, o, v), np.complex128)
    for k in range(N):
        f_oo[k] = np.diag(eo[k])
        f_vv[k] = np.diag(ev[k])
    if spec.fock_offdiag > 0:
        rng2 = np.random.default_rng([spec.seed, 29])
        m = o + v
        P = rng2.standard_normal((N, m, m)) + 1j * rng2.standard_normal((N, m, m))
        P = 0.5 * (P + np.conj(P.transpose(0, 2, 1)))
        if spec.time_reversal:
            for k in range(N):
                if neg[k] < k:
                    P[k] = np.conj(P[neg[k]])
                elif neg[k] == k:
                    P[k] = P[k].real
        for k in range(N):
            np.fill_diagonal(P[k], 0.0)
        P *= spec.fock_offdiag
        f_oo += P[:, :o, :o]
        f_vv += P[:, o:, o:]
        f_ov += P[:, :o, o:]
    return f_oo, f_vv, f_ov


def generate(spec: SynthSpec, blocks=STORED_BLOCKS) -> dict:
    """All inputs of one CCSD problem as a dict of C-contiguous numpy arrays."""
    ks = _ks_table(spec.grid)
    f_oo, f_vv, f_ov = generate_fock(spec)
    out = {"f_oo": f_oo, "f_vv": f_vv, "f_ov": f_ov}
    dt = np.complex64 if spec.int_dtype == "c64" else np.complex128
    for b in blocks:
        H = _block(spec, b, ks)
        out[b] = np.ascontiguousarray(H.astype(dt, copy=False))
        del H
    return out


# ----------------------------------------------- real-space supercell (tests)
def realspace_supercell(spec: SynthSpec):
    """The same Hamiltonian in the localized basis chi_{p R}, built in real space.

    Returns (V, f) with combined index (R, p) -> R * nb + p (p < o occupied):
      V[(R1 p), (R2 q), (R3 r), (R4 s)] = <chi chi || chi chi>  (M^4, M = N nb)
      f[(R p), (R' q)] = N^{-1} sum_k exp(i k.(R - R')) f_k[p, q]
    Only for small cases (dense M^4 storage)."""
    o, v, N = spec.nocc, spec.nvir, spec.nk
    nb = o + v
    cls_of = ["o"] * o + ["v"] * v
    off = {"o": 0, "v": o}
    G = np.zeros((nb, N, nb, N, nb, N, nb), np.complex128)
    for cls in (a + b + c + d for a in "ov" for b in "ov" for c in "ov" for d in "ov"):
        n = {"o": o, "v": v}
        for p in range(n[cls[0]]):
            g = _draw_slice(spec, cls, p)
            G[off[cls[0]] + p, :, off[cls[1]]:off[cls[1]] + n[cls[1]], :,
              off[cls[2]]:off[cls[2]] + n[cls[2]], :,
              off[cls[3]]:off[cls[3]] + n[cls[3]]] = g
    d = _cell_diff(spec.grid)
    M = N * nb
    V = np.zeros((N, nb, N, nb, N, nb, N, nb), np.complex128)
    for R1 in range(N):
        for R2 in range(N):
            for R3 in range(N):
                for R4 in range(N):
                    V[R1, :, R2, :, R3, :, R4, :] = G[:, d[R1, R4], :, d[R2, R4], :, d[R3, R4], :]
    V = V.reshape(M, M, M, M)
    A = V - V.transpose(1, 0, 2, 3) - V.transpose(0, 1, 3, 2) + V.transpose(1, 0, 3, 2)
    H = 0.5 * (A + np.conj(A.transpose(2, 3, 0, 1))) * _scale(spec)
    f_oo, f_vv, f_ov = generate_fock(spec)
    fk = np.zeros((N, nb, nb), np.complex128)
    fk[:, :o, :o] = f_oo
    fk[:, o:, o:] = f_vv
    fk[:, :o, o:] = f_ov
    fk[:, o:, :o] = np.conj(f_ov.transpose(0, 2, 1))
    U = bloch_unitary(spec.grid, nb)        # U[(R p), (k p)]
    F = np.zeros((N * nb, N * nb), np.complex128)
    for k in range(N):
        F[k * nb:(k + 1) * nb, k * nb:(k + 1) * nb] = fk[k]
    f = U @ F @ np.conj(U.T)
    return H, f


def bloch_unitary(grid, nb):
    """U[(R p), (k p')] = delta_{p p'} N^{-1/2} exp(i k.R); columns are the Bloch orbitals."""
    phi = _phase(grid)                      # exp(-i k.R) [k, R]
    N = phi.shape[0]
    U = np.zeros((N, nb, N, nb), np.complex128)
    for p in range(nb):
        U[:, p, :, p] = np.conj(phi).T / math.sqrt(N)
    return U.reshape(N * nb, N * nb)


# ----------------------------------------------------- random amplitudes
def random_amplitudes(spec: SynthSpec, seed: int, scale: float = 0.05):
    """Random antisymmetric, k-conserving t1 (N,o,v) and t2 (N,N,N,o,o,v,v).

    Used to compare residual evaluations at unconverged amplitudes."""
    N, o, v = spec.nk, spec.nocc, spec.nvir
    rng = np.random.default_rng([seed, 31])
    t1 = scale * (rng.standard_normal((N, o, v)) + 1j * rng.standard_normal((N, o, v)))
    x = scale * (rng.standard_normal((N, N, N, o, o, v, v))
                 + 1j * rng.standard_normal((N, N, N, o, o, v, v)))
    ks = _ks_table(spec.grid)
    kk = np.arange(N)
    KI, KJ, KA = np.meshgrid(kk, kk, kk, indexing="ij")
    KB = ks[KI, KJ, KA]
    # antisymmetrize: t[ki,kj,ka](ijab) - t[kj,ki,ka](jiab) - t[ki,kj,kb](ijba) + t[kj,ki,kb](jiba)
    t2 = (x - x[KJ, KI, KA].transpose(0, 1, 2, 4, 3, 5, 6)
          - x[KI, KJ, KB].transpose(0, 1, 2, 3, 4, 6, 5)
          + x[KJ, KI, KB].transpose(0, 1, 2, 4, 3, 6, 5)) * 0.5
    return np.ascontiguousarray(t1), np.ascontiguousarray(t2)


# ------------------------------------------------ torch evaluation (large grids)
# generate() holds every Bloch-transformed class tensor and its antisymmetrized
# copy in host memory, about four times the stored blocks: too much for the
# 3x3x3 grid with 24 virtuals (vvvv alone is 52 GB as complex64).  The same
# recipe evaluated with torch (on a GPU, or on the CPU for the tests that pin it
# to generate()) keeps only the Bloch-transformed classes of one block and its
# result, and forms the antisymmetrized, Hermitized block row by row.  The raw
# draws are the same numpy streams (_draw_slice), so the results agree with
# generate() to the rounding of the FFTs.

def _gk_torch(spec: SynthSpec, cls: str, torch, device):
    n = {"o": spec.nocc, "v": spec.nvir}
    N = spec.nk
    g3 = tuple(spec.grid)
    out = torch.empty((N, N, N, n[cls[0]], n[cls[1]], n[cls[2]], n[cls[3]]), dtype=torch.complex128,
                      device=device)
    fft_dims = (0, 1, 2, 4, 5, 6)
    ifft_dims = (8, 9, 10)
    workers = min(n[cls[0]], os.cpu_count() or 1, 16)
    with ThreadPoolExecutor(max(workers, 1)) as ex:
        futs = [ex.submit(_draw_slice, spec, cls, p) for p in range(n[cls[0]])]
        for p, f in enumerate(futs):
            g = f.result()                                     # (R1, q, R2, r, R3, s)
            nq, nr, ns = g.shape[1], g.shape[3], g.shape[5]
            x = torch.from_numpy(g).to(device).reshape(g3 + (nq,) + g3 + (nr,) + g3 + (ns,))
            del g
            x = torch.fft.fftn(x, dim=fft_dims)
            x = torch.fft.ifftn(x, dim=ifft_dims, norm="forward")
            x = x.reshape(N, nq, N, nr, N, ns)
            out[:, :, :, p] = x.permute(0, 2, 4, 1, 3, 5)
            del x
    out *= 1.0 / N
    return out


def _block_torch(spec: SynthSpec, cls: str, ks, torch, device, out_dtype):
    """One stored block: A = G - G(bra swap) - G(ket swap) + G(both) in k space,
    H = (A + A^dagger) / 2 scaled, formed one (kp, kq) row of blocks at a time."""
    N = spec.nk
    names = {"g0": cls, "gb": _swap(cls, (1, 0, 2, 3)), "gk": _swap(cls, (0, 1, 3, 2)),
             "gbk": _swap(cls, (1, 0, 3, 2))}
    hc = _swap(cls, (2, 3, 0, 1))
    hnames = {"g0": hc, "gb": _swap(hc, (1, 0, 2, 3)), "gk": _swap(hc, (0, 1, 3, 2)),
              "gbk": _swap(hc, (1, 0, 3, 2))}
    cache = {}
    for c in list(names.values()) + list(hnames.values()):
        if c not in cache:
            cache[c] = _gk_torch(spec, c, torch, device)
    ksd = torch.as_tensor(ks, dtype=torch.long, device=device)
    ar = torch.arange(N, device=device)
    sc = 0.5 * _scale(spec)

    def antisym(nm, x, y, z):
        # A_cls[x, y, z] for index tensors of one shape (ks implied), as in _antisym
        kz = ksd[x, y, z]
        a = cache[nm["g0"]][x, y, z] - cache[nm["gb"]][y, x, z].transpose(-4, -3)
        a = a - cache[nm["gk"]][x, y, kz].transpose(-2, -1)
        a = a + cache[nm["gbk"]][y, x, kz].transpose(-4, -3).transpose(-2, -1)
        return a

    shape = cache[cls].shape
    out = torch.empty(shape, dtype=out_dtype, device=device)
    for kp in range(N):
        for kq in range(N):
            xp = torch.full((N,), kp, device=device, dtype=torch.long)
            xq = torch.full((N,), kq, device=device, dtype=torch.long)
            A = antisym(names, xp, xq, ar)                     # [kp, kq, kr] over kr
            kz = ksd[kp, kq]                                   # ks for each kr
            Ah = antisym(hnames, ar, kz, xp)                   # A_h[kr, ks, kp]
            h = A + torch.conj(Ah).permute(0, 3, 4, 1, 2)
            h *= sc
            out[kp, kq] = h.to(out_dtype)
    cache.clear()
    return out


def generate_torch(spec: SynthSpec, device="cuda", blocks=STORED_BLOCKS) -> dict:
    """generate() evaluated with torch on `device`: a dict of contiguous torch
    tensors there (Fock blocks complex128, integral blocks complex128 or, for
    int_dtype "c64", complex64)."""
    import torch
    ks = _ks_table(spec.grid)
    f_oo, f_vv, f_ov = generate_fock(spec)
    out = {"f_oo": torch.from_numpy(f_oo).to(device), "f_vv": torch.from_numpy(f_vv).to(device),
           "f_ov": torch.from_numpy(f_ov).to(device)}
    dt = torch.complex64 if spec.int_dtype == "c64" else torch.complex128
    # largest last: the peak is the vvvv classes plus the smaller results
    for b in sorted(blocks, key=lambda c: c.count("v")):
        out[b] = _block_torch(spec, b, ks, torch, device, dt).contiguous()
        if str(device).startswith("cuda"):
            torch.cuda.empty_cache()
    return out


# ----------------------------------------- random amplitudes, one stream per k_i
def _amp_draws(spec: SynthSpec, seed: int, ki: int, scale: float):
    N, o, v = spec.nk, spec.nocc, spec.nvir
    rng = np.random.default_rng([seed, 37, ki])
    shape = (N, N, o, o, v, v)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def _t1_draws(spec: SynthSpec, seed: int, scale: float):
    N, o, v = spec.nk, spec.nocc, spec.nvir
    rng = np.random.default_rng([seed, 31])
    return scale * (rng.standard_normal((N, o, v)) + 1j * rng.standard_normal((N, o, v)))


def random_amplitudes_slabs(spec: SynthSpec, seed: int, scale: float = 0.05):
    """Random antisymmetric, k-conserving t1 and t2 like random_amplitudes(), drawn
    one k_i slab per stream so that the torch twin below can fill large grids
    quickly; t2 = (x - x(i<->j) - x(a<->b) + x(both)) / 2."""
    N = spec.nk
    t1 = _t1_draws(spec, seed, scale)
    x = np.stack([_amp_draws(spec, seed, ki, scale) for ki in range(N)])
    ks = _ks_table(spec.grid)
    kk = np.arange(N)
    KI, KJ, KA = np.meshgrid(kk, kk, kk, indexing="ij")
    KB = ks[KI, KJ, KA]
    t2 = (x - x[KJ, KI, KA].transpose(0, 1, 2, 4, 3, 5, 6)
          - x[KI, KJ, KB].transpose(0, 1, 2, 3, 4, 6, 5)
          + x[KJ, KI, KB].transpose(0, 1, 2, 4, 3, 6, 5)) * 0.5
    return np.ascontiguousarray(t1), np.ascontiguousarray(t2)


def random_amplitudes_torch(spec: SynthSpec, seed: int, device="cuda", scale: float = 0.05):
    """random_amplitudes_slabs() evaluated with torch on `device` (same draws)."""
    import torch
    N = spec.nk
    t1 = torch.from_numpy(_t1_draws(spec, seed, scale)).to(device)
    x = torch.empty((N, N, N, spec.nocc, spec.nocc, spec.nvir, spec.nvir), dtype=torch.complex128,
                    device=device)
    workers = min(N, os.cpu_count() or 1, 16)
    with ThreadPoolExecutor(max(workers, 1)) as ex:
        for ki, a in enumerate(ex.map(lambda k: _amp_draws(spec, seed, k, scale), range(N))):
            x[ki] = torch.from_numpy(a).to(device)
    ks = torch.as_tensor(_ks_table(spec.grid), dtype=torch.long, device=device)
    t2 = torch.empty_like(x)
    ar = torch.arange(N, device=device)
    for ki in range(N):
        # one k_i slab at a time: x[kj, ki, ka], x[ki, kj, kb], x[kj, ki, kb]
        KJ, KA = torch.meshgrid(ar, ar, indexing="ij")
        KI = torch.full_like(KJ, ki)
        KB = ks[KI, KJ, KA]
        y = x[ki] - x[KJ, KI, KA].transpose(-4, -3) - x[KI, KJ, KB].transpose(-2, -1) \
            + x[KJ, KI, KB].transpose(-4, -3).transpose(-2, -1)
        t2[ki] = y * 0.5
    return t1.contiguous(), t2.contiguous()
