"""Momentum arithmetic on a regular Gamma-centred k grid (paper Sec. 3.2.5).

k points are integer triples (k1, k2, k3), 0 <= kd < nd, flattened as
(k1 * n2 + k2) * n3 + k3.  Momentum equivalence is equality modulo the
reciprocal lattice, i.e. componentwise modulo nd.
"""
import numpy as np


class KMesh:
    def __init__(self, grid):
        self.grid = tuple(int(x) for x in grid)
        n1, n2, n3 = self.grid
        self.nk = n1 * n2 * n3
        idx = np.arange(self.nk)
        self.coords = np.stack([idx // (n2 * n3), (idx // n3) % n2, idx % n3], 1)

    def index(self, c):
        n1, n2, n3 = self.grid
        return int(((c[0] % n1) * n2 + (c[1] % n2)) * n3 + (c[2] % n3))

    def add(self, a, b):
        return self.index(self.coords[a] + self.coords[b])

    def sub(self, a, b):
        return self.index(self.coords[a] - self.coords[b])

    def neg(self, a):
        return self.index(-self.coords[a])

    def k4(self, k1, k2, k3):
        """The fourth momentum fixed by k1 + k2 = k3 + k4."""
        return self.index(self.coords[k1] + self.coords[k2] - self.coords[k3])

    def __iter__(self):
        return iter(range(self.nk))
