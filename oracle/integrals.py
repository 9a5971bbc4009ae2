"""Any class of antisymmetrized integrals from the six stored blocks.

The stored blocks are oooo, ooov, oovv, ovvo, ovvv, vvvv, each laid out as
B[kp][kq][kr][p][q][r][s] with ks = kp + kq - kr.  Every other class follows
from the symmetries the paper states in Sec. 3.3:
    <pq||rs> = <rs||pq>^*                           (Hermiticity)
    <pq||rs> = -<qp||rs> = -<pq||sr> = <qp||sr>     (antisymmetry)
Together they form a group of eight operations on the four slots.
"""
import numpy as np

from .kmesh import KMesh

# (m, sign, conj): the source element is <p_{m0} p_{m1} || p_{m2} p_{m3}>, and
# <p0 p1 || p2 p3> = sign * (conj if conj) of it.
_OPS = (
    ((0, 1, 2, 3), +1, False),
    ((1, 0, 2, 3), -1, False),
    ((0, 1, 3, 2), -1, False),
    ((1, 0, 3, 2), +1, False),
    ((2, 3, 0, 1), +1, True),
    ((3, 2, 0, 1), -1, True),
    ((2, 3, 1, 0), -1, True),
    ((3, 2, 1, 0), +1, True),
)


class Integrals:
    STORED = ("oooo", "ooov", "oovv", "ovvo", "ovvv", "vvvv")

    def __init__(self, blocks: dict, km: KMesh):
        self.b = {k: blocks[k] for k in self.STORED}
        self.km = km

    def get(self, cls: str, kp: int, kq: int, kr: int) -> np.ndarray:
        """Orbital block <p kp q kq || r kr s ks> for slot classes cls, ks implied."""
        ks = self.km.k4(kp, kq, kr)
        k = (kp, kq, kr, ks)
        for m, sign, cj in _OPS:
            src = "".join(cls[j] for j in m)
            if src in self.b:
                sk = [k[j] for j in m]
                S = self.b[src][sk[0], sk[1], sk[2]]
                inv = [0, 0, 0, 0]
                for j in range(4):
                    inv[m[j]] = j
                X = S.transpose(inv)
                if cj:
                    X = np.conj(X)
                return sign * X if sign < 0 else X.copy()
        raise KeyError(cls)
