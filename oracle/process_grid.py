"""The paper's parallel schedule on emulated host ranks (test infrastructure only).

N_k^2 ranks; rank (alpha, beta) has number alpha + beta N_k (paper Sec. 3.2.1).
Every rank runs the same program on its own data and exchanges data only
through the communication procedures of Sec. 4.3:

  reduce_diag      sums over a row or a column into the diagonal rank  (Sec. 4.3.2)
  bcast_vertical,  share F~ from the diagonal ranks with every rank    (Sec. 4.4.2)
  allgather_horizontal
  alltoall         change of the momentum carried by the rank number    (Sec. 4.3.3)
  shift            one step of the Delta loop of the summation of two
                   eight-index quantities ("Sum_88")                     (Sec. 4.3.4)
  diag_swap        exchange of the first and second rank index         (Sec. 4.3.5)

Data placement follows Sec. 3.2: the Fock blocks and R1 on the diagonal
ranks, t1 on every rank, t2[ki][kj][ka] on rank (ki, ka), and the integrals as
Table 1 distributes them (several copies of some classes).  Every integral
block a rank reads is checked against Table 1: a read of a block the rank
does not hold raises LocalityError.  The arithmetic is that of the rearranged
equations (oracle/ccsd_k_rearranged.py: Eqs. EqSingle, EqDouble with A-bar,
A-check, A-tilde, A-hat), step by step in the order of Sec. 4.4.

Two transports run the same program: ThreadComm (one thread per rank in this
process) and GlooComm (one torch.distributed process per rank).  Both count
the bytes every procedure moves between ranks.
"""
import pickle
import threading

import numpy as np

from .integrals import _OPS
from .kmesh import KMesh


def ein(*args):
    return np.einsum(*args, optimize=True)


class LocalityError(RuntimeError):
    pass


# ------------------------------------------------------------- Table 1
# stored class -> owners of block <p kA q kB || r kC s kD> as functions of the
# four momenta; classes listed twice or three times are held in several copies
TABLE1 = {
    "oooo": (lambda a, b, c, d: (c, d),),
    "ooov": (lambda a, b, c, d: (a, c), lambda a, b, c, d: (c, d)),
    "oovv": (lambda a, b, c, d: (a, b), lambda a, b, c, d: (a, c), lambda a, b, c, d: (c, d)),
    "ovvo": (lambda a, b, c, d: (d, b),),
    "ovvv": (lambda a, b, c, d: (a, b), lambda a, b, c, d: (b, d)),
    "vvvv": (lambda a, b, c, d: (a, b),),
}


def _nbytes(x):
    if isinstance(x, np.ndarray):
        return x.nbytes
    if isinstance(x, dict):
        return sum(_nbytes(v) for v in x.values())
    if isinstance(x, (list, tuple)):
        return sum(_nbytes(v) for v in x)
    return 0


# ------------------------------------------------------------- transports
class _CommBase:
    """Collective procedures on top of one primitive: exchange(outgoing) where
    outgoing maps destination rank number -> payload, and every rank calls it
    together; it returns source rank number -> payload."""

    def __init__(self, N):
        self.N = N
        self.stats = {}

    def _count(self, name, rank, outgoing):
        b = sum(_nbytes(v) for d, v in outgoing.items() if d != rank)
        m = sum(1 for d in outgoing if d != rank)
        s = self.stats.setdefault(name, [0, 0])
        s[0] += b
        s[1] += m

    def rid(self, a, b):
        return a + b * self.N

    def reduce_diag(self, ctx, direction, x):
        """Sum over the ranks of a row (horizontal: fixed alpha) or a column
        (vertical: fixed beta) into its diagonal rank; None elsewhere."""
        root = (ctx.alpha, ctx.alpha) if direction == "horizontal" else (ctx.beta, ctx.beta)
        got = self.exchange(ctx, "reduce_" + direction, {self.rid(*root): x})
        if (ctx.alpha, ctx.beta) != root:
            return None
        # fixed order: by the varying rank index
        srcs = sorted(got, key=lambda r: (r // self.N) if direction == "horizontal" else (r % self.N))
        out = None
        for s in srcs:
            out = got[s].copy() if out is None else out + got[s]
        return out

    def bcast_vertical(self, ctx, x):
        """From the diagonal rank (beta, beta) to every rank (alpha, beta)."""
        out = {}
        if ctx.alpha == ctx.beta:
            out = {self.rid(a, ctx.beta): x for a in range(self.N)}
        got = self.exchange(ctx, "bcast_vertical", out)
        return got[self.rid(ctx.beta, ctx.beta)]

    def allgather_horizontal(self, ctx, x):
        """Every rank (alpha, b) of a row contributes x; returns {b: x_b}."""
        got = self.exchange(ctx, "allgather_horizontal", {self.rid(ctx.alpha, b): x for b in range(self.N)})
        return {r // self.N: v for r, v in got.items()}

    def alltoall(self, ctx, direction, outgoing):
        """Index change: outgoing maps the varying rank index (beta for horizontal,
        alpha for vertical) to a payload; returns {varying index: payload}."""
        if direction == "horizontal":
            o = {self.rid(ctx.alpha, b): v for b, v in outgoing.items()}
        else:
            o = {self.rid(a, ctx.beta): v for a, v in outgoing.items()}
        got = self.exchange(ctx, "alltoall_" + direction, o)
        return {(r // self.N if direction == "horizontal" else r % self.N): v for r, v in got.items()}

    def shift(self, ctx, dst, payload):
        """One Delta step of Sum_88: send payload to rank dst = (a, b), receive the
        one payload sent to this rank."""
        got = self.exchange(ctx, "sum88_shift", {self.rid(*dst): payload})
        assert len(got) == 1, "a Sum_88 step must be a permutation of the ranks"
        return next(iter(got.values()))

    def diag_swap(self, ctx, payload):
        """Send to rank (beta, alpha), receive from it (diagonal ranks keep theirs)."""
        got = self.exchange(ctx, "diag_swap", {self.rid(ctx.beta, ctx.alpha): payload})
        return got[self.rid(ctx.beta, ctx.alpha)]

    def gather_all(self, ctx, payload, root=0):
        """Collect payloads on one rank (result extraction, not part of the schedule)."""
        got = self.exchange(ctx, "gather_results", {root: payload})
        return got if ctx.rank == root else None

    def allreduce_max(self, ctx, x):
        got = self.exchange(ctx, "allreduce_max", {r: x for r in range(self.N * self.N)})
        return max(got.values())


class ThreadComm(_CommBase):
    """All ranks as threads of this process, synchronised by a barrier."""

    def __init__(self, N):
        super().__init__(N)
        self.R = N * N
        self.barrier = threading.Barrier(self.R)
        self.lock = threading.Lock()
        self.box = {}

    def exchange(self, ctx, name, outgoing):
        seq = ctx.seq
        ctx.seq += 1
        with self.lock:
            self._count(name, ctx.rank, outgoing)
            for d, v in outgoing.items():
                self.box[(seq, d, ctx.rank)] = v
        self.barrier.wait()
        with self.lock:
            keys = [k for k in self.box if k[0] == seq and k[1] == ctx.rank]
            got = {k[2]: self.box.pop(k) for k in keys}
        self.barrier.wait()
        return got


class GlooComm(_CommBase):
    """One torch.distributed (gloo) process per rank; point-to-point messages are
    exchanged pair by pair in one global order, so no two ranks wait on each other."""

    def __init__(self, N, dist):
        super().__init__(N)
        self.dist = dist

    def exchange(self, ctx, name, outgoing):
        dist = self.dist
        self._count(name, ctx.rank, outgoing)
        dsts = [None] * (self.N * self.N)
        dist.all_gather_object(dsts, sorted(outgoing))
        got = {}
        for s in range(self.N * self.N):
            for d in dsts[s]:
                if s == ctx.rank and d == ctx.rank:
                    got[s] = outgoing[d]
                elif s == ctx.rank:
                    data = np.frombuffer(pickle.dumps(outgoing[d]), dtype=np.uint8)
                    import torch
                    dist.send(torch.tensor([data.size], dtype=torch.int64), dst=d)
                    dist.send(torch.from_numpy(data.copy()), dst=d)
                elif d == ctx.rank:
                    import torch
                    n = torch.zeros(1, dtype=torch.int64)
                    dist.recv(n, src=s)
                    buf = torch.empty(int(n.item()), dtype=torch.uint8)
                    dist.recv(buf, src=s)
                    got[s] = pickle.loads(buf.numpy().tobytes())
        return got


# ------------------------------------------------------------- rank context
class Rank:
    """What one rank holds: t1, its t2 blocks, its integral blocks (through
    Table 1), and on the diagonal its Fock blocks."""

    def __init__(self, alpha, beta, grid, nocc, nvir, arrays, comm):
        self.km = KMesh(grid)
        self.N, self.o, self.v = self.km.nk, nocc, nvir
        self.alpha, self.beta = alpha, beta
        self.rank = alpha + beta * self.N
        self.comm = comm
        self.seq = 0
        self._arr = arrays                    # the input arrays; reads are checked below
        self.diag = alpha == beta

    # integral block of any class, if this rank holds its stored block (Table 1)
    def I(self, cls, kp, kq, kr):
        ks = self.km.k4(kp, kq, kr)
        k = (kp, kq, kr, ks)
        for m, sign, cj in _OPS:
            src = "".join(cls[j] for j in m)
            if src in TABLE1:
                sk = [k[j] for j in m]
                if not any(f(*sk) == (self.alpha, self.beta) for f in TABLE1[src]):
                    raise LocalityError(f"rank {(self.alpha, self.beta)} holds no copy of {src}{tuple(sk)}")
                S = np.asarray(self._arr[src][sk[0], sk[1], sk[2]], np.complex128)
                inv = [0, 0, 0, 0]
                for j in range(4):
                    inv[m[j]] = j
                X = S.transpose(inv)
                if cj:
                    X = np.conj(X)
                return -X if sign < 0 else X.copy()
        raise KeyError(cls)

    def fock(self, name, k):
        if not (self.diag and k == self.alpha):
            raise LocalityError(f"rank {(self.alpha, self.beta)} holds no Fock block of k = {k}")
        return np.asarray(self._arr[name][k], np.complex128)


# ------------------------------------------------------------- the schedule
def residual_program(rk: Rank, t1, T):
    """One evaluation of the right-hand sides on rank rk.

    T: this rank's t2 blocks {(ki, kj, ka): block} with (ki, ka) = (alpha, beta).
    Returns (R1 block on a diagonal rank or None, {(ki, kj, ka): R2 block}) with the
    R2 blocks of this rank (ki = alpha, ka = beta)."""
    N, km, comm = rk.N, rk.km, rk.comm
    a_, b_ = rk.alpha, rk.beta
    k4 = km.k4
    o, v = rk.o, rk.v
    R = range(N)

    # ---- Sec. 4.4.2: F~.  Z~ sums (Sec. 4.3.2), K~ and F~ on the diagonal, then shared
    zoo = np.zeros((o, o), np.complex128)          # Z~_pq^{ke} at (kbar, ke) = (alpha, beta)
    for kn in R:
        zoo += 0.5 * ein("qnef,pnef->pq", T[(a_, kn, b_)], rk.I("oovv", a_, kn, b_))
    zvv = np.zeros((v, v), np.complex128)          # Z~_{km}^gh at (km, kbar) = (alpha, beta)
    for kn in R:
        zvv += 0.5 * ein("mngf,mnhf->gh", T[(a_, kn, b_)], rk.I("oovv", a_, kn, b_))
    zoo_sum = comm.reduce_diag(rk, "horizontal", zoo)
    zvv_sum = comm.reduce_diag(rk, "vertical", zvv)
    Fk = None
    if rk.diag:
        k = a_
        K = np.zeros((o, v), np.complex128)
        for kh in R:
            K += ein("rc,xryc->xy", t1[kh], rk.I("oovv", k, kh, k))
        f_ov = rk.fock("f_ov", k)
        Foo = rk.fock("f_oo", k) + 0.5 * ein("qc,pc->pq", t1[k], f_ov + K) + zoo_sum
        Fvv = rk.fock("f_vv", k) - 0.5 * ein("rg,rh->gh", t1[k], f_ov + K) - zvv_sum
        for kh in R:
            Foo += ein("rc,prqc->pq", t1[kh], rk.I("ooov", k, kh, k))
            Fvv += ein("rc,rgch->gh", t1[kh], rk.I("ovvv", kh, k, kh))
        Fk = (Foo, Fvv, f_ov + K, f_ov)
    Fk = comm.bcast_vertical(rk, Fk)               # rank (alpha, beta) now has F~ of k = beta
    F = comm.allgather_horizontal(rk, Fk)          # and then F~ of every k
    Foo = {k: F[k][0] for k in R}
    Fvv = {k: F[k][1] for k in R}
    Fov = {k: F[k][2] for k in R}

    # ---- Sec. 4.4.3: R1 on the diagonal, with the L~ sums of Sec. 4.3.2
    loo = np.zeros((o, v), np.complex128)          # L~_{p km}^g at (km, kbar) = (alpha, beta)
    for kn in R:
        loo += 0.5 * ein("mngf,mnpf->pg", T[(a_, kn, b_)], rk.I("ooov", a_, kn, b_))
    lvv = np.zeros((o, v), np.complex128)          # L~_p^{g ke} at (kbar, ke) = (alpha, beta)
    for kn in R:
        kf = k4(a_, kn, b_)
        lvv += 0.5 * ein("pnef,ngfe->pg", T[(a_, kn, b_)], rk.I("ovvv", kn, a_, kf))
    loo_sum = comm.reduce_diag(rk, "vertical", loo)
    lvv_sum = comm.reduce_diag(rk, "horizontal", lvv)
    R1 = None
    if rk.diag:
        k = a_
        R1 = np.conj(F[k][3]).copy()
        R1 += ein("pc,gc->pg", t1[k], Fvv[k])
        R1 -= ein("rg,rp->pg", t1[k], Foo[k])
        for kh in R:
            R1 += ein("pngf,nf->pg", T[(k, kh, k)], Fov[kh])
            R1 += ein("rc,rgcp->pg", t1[kh], rk.I("ovvo", kh, k, kh))
        R1 += lvv_sum - loo_sum

    # ---- Sec. 4.4.4: W~_jn^bf on rank (kj, kb)
    # t2 index change (Sec. 4.3.3): t2[kj][ky][kx] from (kj, kx) to (kj, kb), kb = kj + ky - kx
    out = {}
    for ky in R:
        out.setdefault(k4(a_, ky, b_), {})[(a_, ky, b_)] = T[(a_, ky, b_)]
    T_jb = {}
    for blocks in comm.alltoall(rk, "horizontal", out).values():
        T_jb.update(blocks)
    kj, kb = a_, b_
    W = {kn: np.zeros((o, o, v, v), np.complex128) for kn in R}
    # first term by Sum_88: Psi = <n y||f x> held at (kn, kf) (oovv, [ov] copy)
    for d in R:
        # as receiver (kj, kb): kn = kj + Delta; as sender (kn, kf) = (alpha, beta):
        # the receiver is kj' = kn - Delta, kb' = kf + kj' - kn
        kj_r = (a_ - d) % N
        kb_r = k4(b_, kj_r, a_)
        psi = {ky: rk.I("oovv", a_, ky, b_) for ky in R}
        got = comm.shift(rk, (kj_r, kb_r), psi)
        kn = (kj + d) % N
        for ky in R:
            kx = k4(kj, ky, kb)
            W[kn] -= 0.5 * ein("jyxb,nyfx->jnbf", T_jb[(kj, ky, kx)], got[ky])
    for kn in R:                                   # second term, local
        kf = k4(kn, kb, kj)
        W[kn] += ein("nbfj->jnbf", rk.I("ovvo", kn, kb, kf))
    # third term: J~ on rank (kb, kj) = (alpha, beta), then the diagonal swap
    J = {}
    kb2, kj2 = a_, b_
    for kn in R:
        kf = k4(kn, kb2, kj2)
        j = ein("jc,nbfc->jnbf", t1[kj2], rk.I("ovvv", kn, kb2, kf))
        j -= ein("rb,rnjf->jnbf", t1[kb2], rk.I("ooov", kb2, kn, kj2))
        j -= ein("rb,jc,rncf->jnbf", t1[kb2], t1[kj2], rk.I("oovv", kb2, kn, kj2))
        J[kn] = j
    J = comm.diag_swap(rk, J)
    for kn in R:
        W[kn] += J[kn]

    # ---- Sec. 4.4.5: C~ on rank (ki, ka) by Sum_88 with W~ from (kj, kb), then P(ij)P(ab)
    ki, ka = a_, b_
    C = {}
    for kj_ in R:
        kb_ = k4(ki, kj_, ka)
        C[(ki, kj_, ka)] = np.zeros((o, o, v, v), np.complex128)
    for d in R:
        # receiver (ki, ka): kj = ki + Delta; sender (kj, kb) = (alpha, beta) sends its W
        # to ki' = kj - Delta, ka' = kj + kb - ki'  (its own W is for kj = alpha, kb = beta)
        ki_r = (a_ - d) % N
        ka_r = k4(a_, ki_r, b_)
        got = comm.shift(rk, (ki_r, ka_r), W)
        kj_ = (ki + d) % N
        kb_ = k4(ki, kj_, ka)
        for kn in R:
            C[(ki, kj_, ka)] += ein("inaf,jnbf->ijab", T[(ki, kn, ka)], got[kn])
    for kj_ in R:
        kb_ = k4(ki, kj_, ka)
        C[(ki, kj_, ka)] -= ein("rb,jc,raci->ijab", t1[kb_], t1[kj_], rk.I("ovvo", kb_, ka, kj_))
    # C~ with (a ka) <-> (b kb): from rank (ki, kb), horizontal index change
    # (sent keyed by the receiver's block (ki, kj, ka'), ka' = this rank's kb)
    out = {}
    for kj_ in R:
        kb_ = k4(ki, kj_, ka)
        out.setdefault(kb_, {})[(ki, kj_, kb_)] = C[(ki, kj_, ka)]
    Cab = {}
    for blocks in comm.alltoall(rk, "horizontal", out).values():
        Cab.update(blocks)                           # Cab[(ki, kj, ka)] = C[ki, kj, kb]
    # C~ with (i ki) <-> (j kj): from rank (kj, ka), vertical index change
    out = {}
    for kj_ in R:
        out.setdefault(kj_, {})[(kj_, ki, ka)] = C[(ki, kj_, ka)]
    Cij = {}
    for blocks in comm.alltoall(rk, "vertical", out).values():
        Cij.update(blocks)                           # key (ki, kj, ka) = C[kj, ki, ka] for that block
    # both swaps: vertical index change of the (ab)-swapped copy
    out = {}
    for kj_ in R:
        out.setdefault(kj_, {})[(kj_, ki, ka)] = Cab[(ki, kj_, ka)]
    Cboth = {}
    for blocks in comm.alltoall(rk, "vertical", out).values():
        Cboth.update(blocks)
    S2 = {}
    for kj_ in R:
        key = (ki, kj_, ka)
        S2[key] = (C[key] - Cab[key].transpose(0, 1, 3, 2) - Cij[key].transpose(1, 0, 2, 3)
                   + Cboth[key].transpose(1, 0, 3, 2))

    # ---- Sec. 4.4.6: A-bar = P(ij)P(ab) C~ + <ab||ij> + the t1^4 term
    for kj_ in R:
        S2[(ki, kj_, ka)] += np.conj(rk.I("oovv", ki, kj_, ka))
    # t1^4 term computed on rank (ka, ki) = (alpha, beta), then the diagonal swap
    ka2, ki2 = a_, b_
    t4 = {}
    for kj_ in R:
        kb_ = k4(ki2, kj_, ka2)
        t4[(ki2, kj_, ka2)] = ein("ra,sb,ic,jd,rscd->ijab", t1[ka2], t1[kb_], t1[ki2], t1[kj_],
                                  rk.I("oovv", ka2, kb_, ki2))
    t4 = comm.diag_swap(rk, t4)
    for key, blk in t4.items():
        S2[key] += blk

    # ---- Sec. 4.4.7-4.4.9: A-check on rank (ki, kj)
    # t2 redistributed to (ki, kj) (Sec. 4.4.8; the original distribution is kept)
    out = {}
    for kj_ in R:
        out.setdefault(kj_, {})[(a_, kj_, b_)] = T[(a_, kj_, b_)]
    T_ij = {}
    for blocks in comm.alltoall(rk, "horizontal", out).values():
        T_ij.update(blocks)
    ki, kj = a_, b_
    Sc = {}                                          # S2-check, keyed (ki, kj, ka)
    Gc = {}
    for ka_ in R:
        kb_ = k4(ki, kj, ka_)
        eta = ein("ra,sb->rsab", t1[ka_], t1[kb_])
        Sc[(ki, kj, ka_)] = ein("rsab,rsij->ijab", eta, rk.I("oooo", ka_, kb_, ki))
        g = ein("rsab,rsic->icab", eta, rk.I("ooov", ka_, kb_, ki))
        g += np.conj(rk.I("ovvv", ki, kj, ka_))
        Gc[(ki, kj, ka_)] = ein("jc,icab->ijab", t1[kj], g)
        Sc[(ki, kj, ka_)] += Gc[(ki, kj, ka_)]
    Gsw = comm.diag_swap(rk, Gc)                     # G-check[kj, ki, ka] from rank (kj, ki)
    for ka_ in R:
        Sc[(ki, kj, ka_)] -= Gsw[(kj, ki, ka_)].transpose(1, 0, 2, 3)
    for ka_ in R:                                    # Fock terms, after the redistribution
        kb_ = k4(ki, kj, ka_)
        fb = Fvv[kb_] - 0.5 * ein("rb,rf->bf", t1[kb_], Fov[kb_])
        fa = Fvv[ka_] - 0.5 * ein("ra,rf->af", t1[ka_], Fov[ka_])
        Sc[(ki, kj, ka_)] += ein("ijaf,bf->ijab", T_ij[(ki, kj, ka_)], fb)
        Sc[(ki, kj, ka_)] -= ein("ijbf,af->ijab", T_ij[(ki, kj, kb_)], fa)
    # Y~^abef on rank (kb, ka) = (alpha, beta): V~, its diagonal swap, then Y~
    kb2, ka2 = a_, b_
    Vt = {ke: ein("rb,raef->abef", t1[kb2], rk.I("ovvv", kb2, ka2, ke)) for ke in R}   # V~[ka, kb, ke]
    Vsw = comm.diag_swap(rk, Vt)                                                      # V~[kb, ka, ke]
    Y = {}
    for ke in R:
        y = Vt[ke] - Vsw[ke].transpose(1, 0, 2, 3)
        y -= rk.I("vvvv", kb2, ka2, ke).transpose(1, 0, 2, 3)
        y -= ein("sb,ra,sref->abef", t1[kb2], t1[ka2], rk.I("oovv", kb2, ka2, ke))
        Y[ke] = 0.5 * y
    # sum_{ke e f} t_ij^ef Y~^abef by Sum_88: Y~[ka, kb, .] comes from rank (kb, ka)
    for d in R:
        # receiver (ki, kj): ka = ki + Delta; sender (kb, ka) = (alpha, beta) sends to
        # ki' = ka - Delta, kj' = ka + kb - ki'
        ki_r = (b_ - d) % N
        kj_r = k4(b_, a_, ki_r)
        got = comm.shift(rk, (ki_r, kj_r), Y)
        ka_ = (ki + d) % N
        for ke in R:
            Sc[(ki, kj, ka_)] += ein("ijef,abef->ijab", T_ij[(ki, kj, ke)], got[ke])
    # S2-check to (ki, ka) (Sec. 4.4.10), horizontal index change
    out = {}
    for ka_ in R:
        out.setdefault(ka_, {})[(ki, kj, ka_)] = Sc[(ki, kj, ka_)]
    for blocks in comm.alltoall(rk, "horizontal", out).values():
        for key, blk in blocks.items():
            S2[key] += blk

    # ---- Sec. 4.4.11-4.4.12: t2 to (kb, ka); X~ on rank (ki, kj)
    out = {}
    for kj_ in R:
        kb_ = k4(a_, kj_, b_)
        out.setdefault(kb_, {})[(a_, kj_, b_)] = T[(a_, kj_, b_)]
    T_ba = {}
    for blocks in comm.alltoall(rk, "vertical", out).values():
        T_ba.update(blocks)                          # t2[ki][kj][ka] with kb = alpha, ka = beta
    ki, kj = a_, b_
    X = {}
    for kmm in R:
        X[kmm] = np.zeros((o, o, o, o), np.complex128)
    for d in R:
        # receiver (ki, kj): km = ki + Delta; sender (km, kn) = (alpha, beta) holds the
        # [oo] copy of <mn||ef> and sends it to ki' = km - Delta, kj' = km + kn - ki'
        ki_r = (a_ - d) % N
        kj_r = k4(a_, b_, ki_r)
        psi = {ke: rk.I("oovv", a_, b_, ke) for ke in R}
        got = comm.shift(rk, (ki_r, kj_r), psi)
        kmm = (ki + d) % N
        for ke in R:
            X[kmm] += ein("ijef,mnef->mnij", T_ij[(ki, kj, ke)], got[ke])

    # ---- Sec. 4.4.14: Y~_mnij on rank (ki, kj): V~, diagonal swap, Y~
    Vo = {}
    for kmm in R:
        kn = k4(ki, kj, kmm)
        Vo[kmm] = ein("jc,mnic->mnij", t1[kj], rk.I("ooov", kmm, kn, ki))     # V~[km, kn, ki]
    Vosw = comm.diag_swap(rk, Vo)                                              # V~[km, kn, kj]
    Yo = {}
    for kmm in R:
        kn = k4(ki, kj, kmm)
        y = Vo[kmm] - Vosw[kmm].transpose(0, 1, 3, 2)
        y += rk.I("oooo", kmm, kn, ki)
        y += ein("ic,jd,mncd->mnij", t1[ki], t1[kj], rk.I("oovv", kmm, kn, ki))
        Yo[kmm] = 0.5 * y

    # ---- Sec. 4.4.13-4.4.16: A-tilde + A-hat on rank (kb, ka)
    kb, ka = a_, b_
    Sh = {}
    for ki_ in R:
        Sh[(ki_, k4(ka, kb, ki_), ka)] = np.zeros((o, o, v, v), np.complex128)
    for d in R:
        # receiver (kb, ka): ki = kb + Delta; sender (ki, kj) = (alpha, beta) sends X~ and
        # Y~_mnij to kb' = ki - Delta, ka' = ki + kj - kb'
        kb_r = (a_ - d) % N
        ka_r = k4(a_, b_, kb_r)
        got = comm.shift(rk, (kb_r, ka_r), (X, Yo))
        ki_ = (kb + d) % N
        kj_ = k4(ka, kb, ki_)
        Xr, Yr = got
        for kmm in R:
            kn = k4(ki_, kj_, kmm)
            Sh[(ki_, kj_, ka)] += 0.25 * ein("mnab,mnij->ijab", T_ba[(kmm, kn, ka)], Xr[kmm])
            Sh[(ki_, kj_, ka)] += ein("mnab,mnij->ijab", T_ba[(kmm, kn, ka)], Yr[kmm])
    Gh = {}
    for ki_ in R:
        kj_ = k4(ka, kb, ki_)
        key = (ki_, kj_, ka)
        fj = Foo[kj_] + 0.5 * ein("jc,nc->nj", t1[kj_], Fov[kj_])
        fi = Foo[ki_] + 0.5 * ein("ic,nc->ni", t1[ki_], Fov[ki_])
        Sh[key] -= ein("inab,nj->ijab", T_ba[(ki_, kj_, ka)], fj)
        Sh[key] += ein("jnab,ni->ijab", T_ba[(kj_, ki_, ka)], fi)
        eta = ein("ic,jd->ijcd", t1[ki_], t1[kj_])
        Sh[key] -= ein("ijcd,bacd->ijab", eta, rk.I("vvvv", kb, ka, ki_))
        g = ein("ijcd,racd->rija", eta, rk.I("ovvv", kb, ka, ki_))
        g += np.conj(rk.I("ooov", ki_, kj_, kb)).transpose(2, 0, 1, 3)
        Gh[key] = ein("rb,rija->ijab", t1[kb], g)
        Sh[key] += Gh[key]
    Ghsw = comm.diag_swap(rk, Gh)                    # G-hat[ki, kj, kb] from rank (ka, kb)
    for ki_ in R:
        kj_ = k4(ka, kb, ki_)
        Sh[(ki_, kj_, ka)] -= Ghsw[(ki_, kj_, kb)].transpose(0, 1, 3, 2)
    # S2-hat to (ki, ka) (Sec. 4.4.17), vertical index change
    out = {}
    for ki_ in R:
        kj_ = k4(ka, kb, ki_)
        out.setdefault(ki_, {})[(ki_, kj_, ka)] = Sh[(ki_, kj_, ka)]
    for blocks in comm.alltoall(rk, "vertical", out).values():
        for key, blk in blocks.items():
            S2[key] += blk
    return R1, S2


def iterate_program(rk: Rank, t1, T, n_iter):
    """n_iter Jacobi updates t <- t + R/D (Sec. 4.4.18-4.4.19) from the given amplitudes,
    each with the global max|R| (the convergence test).  Returns (t1, T, norms)."""
    N, km = rk.N, rk.km
    norms = []
    # the denominators need the Fock diagonals of every k: shared like F~
    d = None
    if rk.diag:
        d = (np.real(np.diag(rk.fock("f_oo", rk.alpha))).copy(), np.real(np.diag(rk.fock("f_vv", rk.alpha))).copy())
    d = rk.comm.bcast_vertical(rk, d)
    D = rk.comm.allgather_horizontal(rk, d)
    eo = {k: D[k][0] for k in range(N)}
    ev = {k: D[k][1] for k in range(N)}
    for _ in range(n_iter):
        R1, S2 = residual_program(rk, t1, T)
        m = max(float(np.abs(b).max()) for b in S2.values())
        if R1 is not None:
            m = max(m, float(np.abs(R1).max()))
        norms.append(rk.comm.allreduce_max(rk, m))
        # t1 update on the diagonal, then shared with every rank
        upd = None
        if R1 is not None:
            k = rk.alpha
            upd = t1[k] + R1 / (eo[k][:, None] - ev[k][None, :])
        upd = rk.comm.bcast_vertical(rk, upd)
        T1 = rk.comm.allgather_horizontal(rk, upd)
        newT = {}
        for (ki, kj, ka), blk in T.items():
            kb = km.k4(ki, kj, ka)
            den = (eo[ki][:, None, None, None] + eo[kj][None, :, None, None]
                   - ev[ka][None, None, :, None] - ev[kb][None, None, None, :])
            newT[(ki, kj, ka)] = blk + S2[(ki, kj, ka)] / den
        t1 = np.stack([T1[k] for k in range(N)])
        T = newT
    return t1, T, norms


# ------------------------------------------------------------- drivers
def local_t2(t2, alpha, beta, N):
    """The t2 blocks rank (alpha, beta) holds: t2[alpha][kj][beta] for every kj."""
    return {(alpha, kj, beta): np.asarray(t2[alpha, kj, beta], np.complex128) for kj in range(N)}


def run_threads(grid, nocc, nvir, arrays, t1, t2, n_iter=0):
    """Run the schedule with one thread per rank.  n_iter = 0: one residual
    evaluation, returns (R1, R2, stats); n_iter > 0: that many updates, returns
    (t1, t2, norms, stats).  Arrays are gathered from their owning ranks."""
    km = KMesh(grid)
    N = km.nk
    comm = ThreadComm(N)
    results = {}
    errors = []

    def body(alpha, beta):
        try:
            rk = Rank(alpha, beta, grid, nocc, nvir, arrays, comm)
            T = local_t2(t2, alpha, beta, N)
            if n_iter == 0:
                results[(alpha, beta)] = residual_program(rk, np.asarray(t1, np.complex128), T)
            else:
                results[(alpha, beta)] = iterate_program(rk, np.asarray(t1, np.complex128), T, n_iter)
        except BaseException as e:       # noqa: BLE001  (re-raised by the caller)
            errors.append(e)
            comm.barrier.abort()

    threads = [threading.Thread(target=body, args=(a, b)) for b in range(N) for a in range(N)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    if errors:
        raise errors[0]
    stats = {k: tuple(v) for k, v in comm.stats.items()}
    if n_iter == 0:
        R1 = np.zeros_like(np.asarray(t1, np.complex128))
        R2 = np.zeros(np.shape(t2), np.complex128)
        for (a, b), (r1, s2) in results.items():
            if r1 is not None:
                R1[a] = r1
            for (ki, kj, ka), blk in s2.items():
                R2[ki, kj, ka] = blk
        return R1, R2, stats
    T1 = results[(0, 0)][0]
    T2 = np.zeros(np.shape(t2), np.complex128)
    for (a, b), (_, T, _) in results.items():
        for (ki, kj, ka), blk in T.items():
            T2[ki, kj, ka] = blk
    return T1, T2, results[(0, 0)][2], stats
