"""Form A residual at selected momentum blocks (test infrastructure only).

For problems too large for ccsd_k.residual (the 3x3x3 grid with 24 virtual
spin orbitals has a 104 GB W~^abef in complex128): R1 at chosen k points and R2
at chosen (ki, kj, ka) blocks, from the same equations -- the T1 residual of
Eq. (ori_EqSingle), the T2 residual of Eq. (ori_EqDouble) with its P(ij),
P(ab), P(ij)P(ab) operators, the intermediates W~_mnij, W~^abef, W~_jn^bf
(Eq. Def_Woovv), F~ (Eqs. ori_F_ov, ori_F_oo, ori_F_vv) and tau, tau~ (Sec. 2)
-- with every intermediate formed only at the momenta the requested blocks
need.  The sums and their order follow ccsd_k term by term; nothing is
regrouped.  Integral blocks may be stored complex64: each block is widened to
complex128 when it is read, so the arithmetic is FP64 throughout.
"""
import numpy as np

from .integrals import Integrals
from .kmesh import KMesh


def ein(*args):
    return np.einsum(*args, optimize=True)


class BlockProblem:
    """Inputs kept as given (numpy arrays of any complex type); blocks are read
    and widened on demand."""

    def __init__(self, grid, nocc, nvir, arrays: dict):
        self.km = KMesh(grid)
        self.nk, self.o, self.v = self.km.nk, nocc, nvir
        self.f_oo = np.asarray(arrays["f_oo"], np.complex128)
        self.f_vv = np.asarray(arrays["f_vv"], np.complex128)
        self.f_ov = np.asarray(arrays["f_ov"], np.complex128)
        self._I = Integrals({k: arrays[k] for k in Integrals.STORED}, self.km)

    def get(self, cls, kp, kq, kr):
        return np.asarray(self._I.get(cls, kp, kq, kr), np.complex128)


class BlockResidual:
    """R1[k] and R2[ki, kj, ka] of form A at amplitudes (t1, t2) (complex128 arrays
    in the library layout).  Intermediates are memoized per momentum block."""

    def __init__(self, P: BlockProblem, t1, t2):
        self.P, self.t1, self.t2 = P, t1, t2
        self._tau = {}
        self._wmnij, self._wabef, self._wring = {}, {}, {}
        self._fock = None

    # tau~ and tau of one block (ccsd_k.taus)
    def taus(self, ki, kj, ka):
        key = (ki, kj, ka)
        if key not in self._tau:
            km, t1 = self.P.km, self.t1
            kb = km.k4(ki, kj, ka)
            x = np.zeros(self.t2.shape[3:], np.complex128)
            if ki == ka:
                x += ein("ia,jb->ijab", t1[ki], t1[kj])
            if ki == kb:
                x -= ein("ib,ja->ijab", t1[ki], t1[kj])
            t = np.asarray(self.t2[ki, kj, ka], np.complex128)
            self._tau[key] = (t + 0.5 * x, t + x)
        return self._tau[key]

    def tau(self, ki, kj, ka):
        return self.taus(ki, kj, ka)[1]

    # F~_ov, F~_oo, F~_vv at every k (ccsd_k.f_*_tilde); tau~ blocks are formed on the
    # fly and not kept
    def fock(self):
        if self._fock is None:
            P, km, t1 = self.P, self.P.km, self.t1
            Fov = P.f_ov.copy()
            Foo = P.f_oo.copy()
            Fvv = P.f_vv.copy()
            for k in km:
                for kh in km:
                    Fov[k] += ein("rc,prgc->pg", t1[kh], P.get("oovv", k, kh, k))
            for k in km:
                Foo[k] += 0.5 * ein("pc,qc->pq", P.f_ov[k], t1[k])
                for kh in km:
                    Foo[k] += ein("rc,prqc->pq", t1[kh], P.get("ooov", k, kh, k))
                for kn in km:
                    for ke in km:
                        tt = self._tau_t_nocache(k, kn, ke)
                        Foo[k] += 0.5 * ein("qnef,pnef->pq", tt, P.get("oovv", k, kn, ke))
            for k in km:
                Fvv[k] -= 0.5 * ein("rh,rg->gh", P.f_ov[k], t1[k])
                for kh in km:
                    Fvv[k] += ein("rc,grhc->gh", t1[kh], P.get("vovv", k, kh, k))
                for kmm in km:
                    for kn in km:
                        tt = self._tau_t_nocache(kmm, kn, k)
                        Fvv[k] -= 0.5 * ein("mngf,mnhf->gh", tt, P.get("oovv", kmm, kn, k))
            Fvv_p = np.empty_like(Fvv)
            Foo_p = np.empty_like(Foo)
            for k in km:
                Fvv_p[k] = Fvv[k] - 0.5 * ein("rb,rf->bf", t1[k], Fov[k])
                Foo_p[k] = Foo[k] + 0.5 * ein("jc,nc->nj", t1[k], Fov[k])
            self._fock = (Fov, Foo, Fvv, Foo_p, Fvv_p)
        return self._fock

    def _tau_t_nocache(self, ki, kj, ka):
        if (ki, kj, ka) in self._tau:
            return self._tau[(ki, kj, ka)][0]
        km, t1 = self.P.km, self.t1
        kb = km.k4(ki, kj, ka)
        x = np.zeros(self.t2.shape[3:], np.complex128)
        if ki == ka:
            x += ein("ia,jb->ijab", t1[ki], t1[kj])
        if ki == kb:
            x -= ein("ib,ja->ijab", t1[ki], t1[kj])
        return np.asarray(self.t2[ki, kj, ka], np.complex128) + 0.5 * x

    # intermediates at one momentum block (ccsd_k.w_mnij, w_abef, w_ring)
    def w_mnij(self, kmm, kn, ki):
        key = (kmm, kn, ki)
        if key not in self._wmnij:
            P, km, t1 = self.P, self.P.km, self.t1
            kj = km.k4(kmm, kn, ki)
            w = P.get("oooo", kmm, kn, ki).copy()
            w += ein("jc,mnic->mnij", t1[kj], P.get("ooov", kmm, kn, ki))
            w -= ein("ic,mnjc->mnij", t1[ki], P.get("ooov", kmm, kn, kj))
            for ke in km:
                w += 0.25 * ein("ijef,mnef->mnij", self.tau(ki, kj, ke), P.get("oovv", kmm, kn, ke))
            self._wmnij[key] = w
        return self._wmnij[key]

    def w_abef(self, ka, kb, ke):
        key = (ka, kb, ke)
        if key not in self._wabef:
            P, km, t1 = self.P, self.P.km, self.t1
            w = P.get("vvvv", ka, kb, ke).copy()
            w -= ein("rb,aref->abef", t1[kb], P.get("vovv", ka, kb, ke))
            w += ein("ra,bref->abef", t1[ka], P.get("vovv", kb, ka, ke))
            for kmm in km:
                kn = km.k4(ka, kb, kmm)
                w += 0.25 * ein("mnab,mnef->abef", self.tau(kmm, kn, ka), P.get("oovv", kmm, kn, ke))
            self._wabef[key] = w
        return self._wabef[key]

    def w_ring(self, kj, kn, kb):
        key = (kj, kn, kb)
        if key not in self._wring:
            P, km, t1, t2 = self.P, self.P.km, self.t1, self.t2
            kf = km.k4(kn, kb, kj)
            w = ein("nbfj->jnbf", P.get("ovvo", kn, kb, kf))
            w += ein("jc,nbfc->jnbf", t1[kj], P.get("ovvv", kn, kb, kf))
            w -= ein("rb,nrfj->jnbf", t1[kb], P.get("oovo", kn, kb, kf))
            for kx in km:
                ky = km.k4(kj, kx, kb)
                w -= 0.5 * ein("jxyb,nxfy->jnbf", t2[kj, kx, ky], P.get("oovv", kn, kx, kf))
            w -= ein("jc,rb,nrfc->jnbf", t1[kj], t1[kb], P.get("oovv", kn, kb, kf))
            self._wring[key] = w
        return self._wring[key]

    # the three groups of T2 terms under P(ab), P(ij), P(ij)P(ab), at one block
    def z_ab(self, ki, kj, ka):
        P, km, t1 = self.P, self.P.km, self.t1
        kb = km.k4(ki, kj, ka)
        Fvv_p = self.fock()[4]
        z = ein("ijaf,bf->ijab", self.t2[ki, kj, ka], Fvv_p[kb])
        z -= ein("ra,rbij->ijab", t1[ka], P.get("ovoo", ka, kb, ki))
        return z

    def z_ij(self, ki, kj, ka):
        P, km, t1 = self.P, self.P.km, self.t1
        kb = km.k4(ki, kj, ka)
        Foo_p = self.fock()[3]
        z = -ein("inab,nj->ijab", self.t2[ki, kj, ka], Foo_p[kj])
        z += ein("abcj,ic->ijab", P.get("vvvo", ka, kb, ki), t1[ki])
        return z

    def z_ijab(self, ki, kj, ka):
        P, km, t1, t2 = self.P, self.P.km, self.t1, self.t2
        kb = km.k4(ki, kj, ka)
        z = np.zeros(t2.shape[3:], np.complex128)
        for kn in km:
            z += ein("inaf,jnbf->ijab", t2[ki, kn, ka], self.w_ring(kj, kn, kb))
        z -= ein("ic,ra,rbcj->ijab", t1[ki], t1[ka], P.get("ovvo", ka, kb, ki))
        return z

    def r1(self, k):
        P, km, t1, t2 = self.P, self.P.km, self.t1, self.t2
        Fov, Foo, Fvv = self.fock()[:3]
        r = np.conj(P.f_ov[k]).copy()
        r += ein("ac,ic->ia", Fvv[k], t1[k])
        r -= ein("ra,ri->ia", t1[k], Foo[k])
        for kh in km:
            r += ein("nf,inaf->ia", Fov[kh], t2[k, kh, k])
            r += ein("rc,aric->ia", t1[kh], P.get("voov", k, kh, k))
        for kmm in km:
            for kn in km:
                r -= 0.5 * ein("mnaf,mnif->ia", t2[kmm, kn, k], P.get("ooov", kmm, kn, k))
        for kn in km:
            for ke in km:
                r += 0.5 * ein("inef,anef->ia", t2[k, kn, ke], P.get("vovv", k, kn, ke))
        return r

    def r2(self, ki, kj, ka):
        P, km = self.P, self.P.km
        kb = km.k4(ki, kj, ka)
        r = np.conj(P.get("oovv", ki, kj, ka))
        for kmm in km:
            kn = km.k4(ki, kj, kmm)
            r += 0.5 * ein("mnab,mnij->ijab", self.tau(kmm, kn, ka), self.w_mnij(kmm, kn, ki))
        for ke in km:
            r += 0.5 * ein("abef,ijef->ijab", self.w_abef(ka, kb, ke), self.tau(ki, kj, ke))
        # P(ab) Zab, P(ij) Zij, P(ij) P(ab) Zijab, each operator swapping momentum and index
        r += self.z_ab(ki, kj, ka) - self.z_ab(ki, kj, kb).transpose(0, 1, 3, 2)
        r += self.z_ij(ki, kj, ka) - self.z_ij(kj, ki, ka).transpose(1, 0, 2, 3)
        r += (self.z_ijab(ki, kj, ka) - self.z_ijab(ki, kj, kb).transpose(0, 1, 3, 2)
              - self.z_ijab(kj, ki, ka).transpose(1, 0, 2, 3)
              + self.z_ijab(kj, ki, kb).transpose(1, 0, 3, 2))
        return r
