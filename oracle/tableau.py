"""CHP stabiliser tableau (Aaronson & Gottesman, Phys. Rev. A 70, 052328 (2004)), test infrastructure.

Used only to pin the state-vector and MPS oracles on Clifford circuits: it decides from the
tableau alone whether a Z measurement is deterministic (and its value) or uniformly random.
Rows 0..n-1 are destabilisers, rows n..2n-1 stabilisers, row 2n is scratch.
"""
from __future__ import annotations

import numpy as np


class Tableau:
    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros(2 * n + 1, dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1
            self.z[n + i, i] = 1

    # -- gates (the paper's update rules for CNOT, H and phase; the rest composed) ---------------
    def cx(self, a, b):
        x, z = self.x, self.z
        self.r ^= x[:, a] & z[:, b] & (x[:, b] ^ z[:, a] ^ 1)
        x[:, b] ^= x[:, a]
        z[:, a] ^= z[:, b]

    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def apply(self, name, qs):
        a = qs[0]
        if name == "H":
            self.h(a)
        elif name == "S":
            self.s(a)
        elif name == "SDG":
            self.s(a); self.s(a); self.s(a)
        elif name == "Z":
            self.r ^= self.x[:, a]
        elif name == "X":
            self.r ^= self.z[:, a]
        elif name == "Y":
            self.r ^= self.x[:, a] ^ self.z[:, a]
        elif name == "CX":
            self.cx(a, qs[1])
        elif name == "CZ":
            self.h(qs[1]); self.cx(a, qs[1]); self.h(qs[1])
        elif name == "SWAP":
            b = qs[1]
            self.cx(a, b); self.cx(b, a); self.cx(a, b)
        else:
            raise ValueError(f"{name} is not a Clifford gate")

    # -- measurement -----------------------------------------------------------------------------
    @staticmethod
    def _g(x1, z1, x2, z2):
        x1, z1, x2, z2 = (v.astype(np.int64) for v in (x1, z1, x2, z2))
        return np.where((x1 == 0) & (z1 == 0), 0,
               np.where((x1 == 1) & (z1 == 1), z2 - x2,
               np.where(x1 == 1, z2 * (2 * x2 - 1), x2 * (1 - 2 * z2))))

    def _rowsum(self, h, i):
        tot = 2 * int(self.r[h]) + 2 * int(self.r[i]) + int(np.sum(
            self._g(self.x[i], self.z[i], self.x[h], self.z[h])))
        self.r[h] = 0 if tot % 4 == 0 else 1
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def peek_z(self, a):
        """(deterministic, value): value is the outcome when deterministic."""
        n = self.n
        if np.any(self.x[n:2 * n, a]):
            return False, None
        s = 2 * n
        self.x[s] = 0
        self.z[s] = 0
        self.r[s] = 0
        for i in range(n):
            if self.x[i, a]:
                self._rowsum(s, i + n)
        return True, int(self.r[s])

    def measure_z(self, a, forced=0):
        """Measure Z on qubit a; a random outcome takes the value `forced`."""
        n = self.n
        ps = np.nonzero(self.x[n:2 * n, a])[0]
        if len(ps) == 0:
            return self.peek_z(a)[1]
        p = int(ps[0]) + n
        for i in range(2 * n):
            if i != p and self.x[i, a]:
                self._rowsum(i, p)
        self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p].copy(), self.z[p].copy(), self.r[p]
        self.x[p] = 0
        self.z[p] = 0
        self.z[p, a] = 1
        self.r[p] = forced
        return forced
