"""Plain FP64, one-shot-per-launch GPU MPS: the comparator of the throughput claim.

This is the straightforward way to run the same computation on a GPU -- one shot at a time,
every gate its own sequence of PyTorch launches, the library SVD (cuSOLVER) for every two-site
split, complex128 throughout -- written only so that the batched engine's throughput can be
compared with it.  It is not part of the sampling path and shares nothing with the CUDA library
except the fault lists, which it takes as input.

Semantics follow the engine: SWAP routing for non-adjacent gates (Sec. 3.1), the truncation rule
(smallest kept count whose discarded tail is <= cutoff, at most chi_max), readouts from the Born
rule with the 53-bit Philox uniforms of the random-number contract, early stop at the first
measurement returning 1 (Sec. 4.3).
"""
from __future__ import annotations

import math

import numpy as np
import torch

_SQ = math.sqrt(0.5)
_W = (0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85)


def _philox(c, k):
    c0, c1, c2, c3 = c
    k0, k1 = k
    for _ in range(10):
        p0 = _W[0] * c0
        p1 = _W[1] * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & 0xFFFFFFFF, p1 & 0xFFFFFFFF, ((p0 >> 32) ^ c3 ^ k1) & 0xFFFFFFFF, \
            p0 & 0xFFFFFFFF
        k0 = (k0 + _W[2]) & 0xFFFFFFFF
        k1 = (k1 + _W[3]) & 0xFFFFFFFF
    return c0, c1, c2, c3


def readout_uniform(seed, k, shot):
    x = _philox((k & 0xFFFFFFFF, shot & 0xFFFFFFFF, shot >> 32, 3), (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    return ((x[0] >> 5) * (1 << 26) + (x[1] >> 6)) / 9007199254740992.0


def _gates(dev):
    c = lambda m: torch.tensor(m, dtype=torch.complex128, device=dev)
    t = complex(math.cos(math.pi / 4), math.sin(math.pi / 4))
    one = {"H": c([[_SQ, _SQ], [_SQ, -_SQ]]), "S": c([[1, 0], [0, 1j]]), "SDG": c([[1, 0], [0, -1j]]),
           "X": c([[0, 1], [1, 0]]), "Y": c([[0, -1j], [1j, 0]]), "Z": c([[1, 0], [0, -1]]),
           "T": c([[1, 0], [0, t]]), "TDG": c([[1, 0], [0, t.conjugate()]])}
    two = {"CX": c([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]]),
           "CZ": c(np.diag([1, 1, 1, -1])),
           "SWAP": c([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]])}
    paulis = [c(np.eye(2)), one["X"], one["Y"], one["Z"]]
    return one, two, paulis


def parse(text):
    ops, n, chan, read = [], 0, 0, 0
    for line in text.splitlines():
        t = line.split("#", 1)[0].split()
        if not t:
            continue
        name = t[0].upper()
        if name == "QUBITS":
            n = int(t[1])
            continue
        if name == "TICK":
            continue
        qs = tuple(int(v) for v in t[1:])
        aux = None
        if name in ("DEP1", "DEP2", "XERR"):
            aux = chan
            chan += 1
        elif name in ("M", "R"):
            aux = read
            read += 1
        ops.append((name, qs, aux))
    return n, ops


class PlainMPS:
    def __init__(self, n, chi_max, cutoff, dev):
        self.n, self.chi, self.cut, self.dev = n, chi_max, cutoff, dev
        self.A = [torch.zeros((1, 2, 1), dtype=torch.complex128, device=dev) for _ in range(n)]
        for a in self.A:
            a[0, 0, 0] = 1
        self.center = 0
        self.updates = 0

    def _move(self, q):
        while self.center < q:
            k = self.center
            a = self.A[k]
            l, d, r = a.shape
            qm, rm = torch.linalg.qr(a.reshape(l * d, r))
            self.A[k] = qm.reshape(l, d, -1)
            self.A[k + 1] = torch.tensordot(rm, self.A[k + 1], dims=([1], [0]))
            self.center += 1
        while self.center > q:
            k = self.center
            a = self.A[k]
            l, d, r = a.shape
            qm, rm = torch.linalg.qr(a.reshape(l, d * r).conj().T)
            self.A[k] = qm.conj().T.reshape(-1, d, r)
            self.A[k - 1] = torch.tensordot(self.A[k - 1], rm.conj().T, dims=([2], [0]))
            self.center -= 1

    def two_site(self, g4, q):
        self._move(q)
        a, b = self.A[q], self.A[q + 1]
        l, r = a.shape[0], b.shape[2]
        th = torch.einsum("lsm,mtr->lstr", a, b)
        th = torch.einsum("stuv,luvr->lstr", g4.reshape(2, 2, 2, 2), th).reshape(2 * l, 2 * r)
        u, s, vh = torch.linalg.svd(th, full_matrices=False)
        s2 = (s * s).cpu().numpy()
        tot = s2.sum()
        tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])
        k = 1
        while k < len(s2) and tail[k] > self.cut * tot:
            k += 1
        k = min(k, self.chi)
        sk = s[:k] / torch.sqrt(torch.sum(s[:k] ** 2))
        self.A[q] = u[:, :k].reshape(l, 2, k)
        self.A[q + 1] = (sk[:, None].to(vh.dtype) * vh[:k]).reshape(k, 2, r)
        self.center = q + 1
        self.updates += 1

    def gate2(self, g4, a, b, sw):
        if abs(a - b) == 1:
            self.two_site(g4 if a < b else sw @ g4 @ sw, min(a, b))
            return
        lo, hi = min(a, b), max(a, b)
        for i in range(lo, hi - 1):
            self.two_site(sw, i)
        self.two_site(g4 if a < b else sw @ g4 @ sw, hi - 1)
        for i in range(hi - 2, lo - 1, -1):
            self.two_site(sw, i)

    def one(self, u, q):
        self.A[q] = torch.einsum("st,ltr->lsr", u, self.A[q])

    def prob1(self, q):
        self._move(q)
        a = self.A[q]
        p = (a.abs() ** 2).sum(dim=(0, 2))
        return float(p[1] / p.sum())

    def project(self, q, o):
        a = self.A[q].clone()
        a[:, 1 - o, :] = 0
        self.A[q] = a / torch.sqrt((a.abs() ** 2).sum())


def run_shot(n, ops, faults, *, seed, shot, chi_max, cutoff, dev, max_updates=None):
    """One shot; returns (status, updates).  faults: dict channel -> pauli code."""
    one, two, paulis = _gates(dev)
    m = PlainMPS(n, chi_max, cutoff, dev)
    sw = two["SWAP"]
    for name, qs, aux in ops:
        if max_updates is not None and m.updates >= max_updates:
            return "cut", m.updates
        if name in one:
            m.one(one[name], qs[0])
        elif name in two:
            m.gate2(two[name], qs[0], qs[1], sw)
        elif name in ("DEP1", "DEP2", "XERR"):
            code = faults.get(aux)
            if code:
                if name == "DEP2":
                    m.one(paulis[code >> 2], qs[0])
                    m.one(paulis[code & 3], qs[1])
                else:
                    m.one(paulis[code], qs[0])
        else:
            q = qs[0]
            p1 = m.prob1(q)
            o = 1 if readout_uniform(seed, aux, shot) < p1 else 0
            if name == "M" and o == 1:
                return "rejected", m.updates
            m.project(q, o)
            if name == "R" and o == 1:
                m.one(one["X"], q)
    if str(dev).startswith("cuda"):
        torch.cuda.synchronize()
    return "accepted", m.updates
