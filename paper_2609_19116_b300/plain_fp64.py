"""Plain FP64, one-shot-per-launch GPU MPS: the comparator of the throughput claim.

This is the straightforward way to run the same computation on a GPU -- one shot at a time,
every gate its own sequence of PyTorch launches, the library SVD (cuSOLVER) for every two-site
split, complex128 throughout -- written only so that the batched engine's throughput can be
compared with it.  It is not part of the sampling path and shares nothing with the CUDA library
except the fault lists, which it takes as input.

Semantics follow the engine: SWAP routing for non-adjacent gates (Sec. 3.1) with the engine's
routing rules (a moved qubit stays where it was moved; the mover is the unentangled qubit, else the
one reset first, else the one whose next partner is nearer; a reset qubit walks home; a logical
SWAP relabels; a SWAP with an unentangled qubit is an exact relabelling of bonds), the truncation
rule (smallest kept count whose discarded tail is <= cutoff, at most chi_max), readouts from the
Born rule with the 53-bit Philox uniforms of the random-number contract, early stop at the first
measurement returning 1 (Sec. 4.3).  Instructions run in text order.
"""
from __future__ import annotations

import bisect
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

    def product_swap(self, k, prod_left):
        """SWAP of sites k, k+1 where one qubit is unentangled: A = phi (x) M, no SVD.  When the
        relabelled bond would be wider than the other side allows (a readout leaves bonds wider
        than the state needs) or the tensor does not show the product form, the SWAP goes
        through the SVD instead (exact either way)."""
        l, r = self.A[k].shape[0], self.A[k + 1].shape[2]
        p = k if prod_left else k + 1
        a = self.A[p]
        rho = torch.einsum("lsr,ltr->st", a, a.conj())
        ev = torch.linalg.eigvalsh(rho)
        # a QR move through a site whose matrix is rank-deficient completes Q with directions
        # outside the qubit's state, so the tensor need not show the product form: use the SVD
        if (prod_left and r > 2 * l) or (not prod_left and l > 2 * r) or float(ev[0]) > 1e-12 * float(ev[1]):
            self.two_site(torch.tensor([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]],
                                       dtype=self.A[k].dtype, device=self.dev), k)
            self.updates -= 1  # counted as the product SWAP it stands for
            return
        s0 = int(torch.argmax(rho.diagonal().real))
        phi = rho[:, s0] / torch.sqrt(rho[s0, s0].real * rho.diagonal().real.sum())
        mm = torch.einsum("s,lsr->lr", phi.conj(), a)
        if prod_left:
            b = self.A[k + 1]
            r = b.shape[2]
            self.A[k] = torch.tensordot(mm, b, dims=([1], [0]))
            self.A[k + 1] = torch.einsum("s,ab->asb", phi, torch.eye(r, dtype=a.dtype, device=self.dev))
            if self.center in (k, k + 1):
                self.center = k
        else:
            b = self.A[k]
            l = b.shape[0]
            self.A[k + 1] = torch.tensordot(b, mm, dims=([2], [0]))
            self.A[k] = torch.einsum("s,ab->asb", phi, torch.eye(l, dtype=a.dtype, device=self.dev))
            if self.center in (k, k + 1):
                self.center = k + 1

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


def plan(n, ops, return_layout=False):
    """Routed steps in text order: ("1q", name, site) | ("ch", name, sites, aux) |
    ("g2", name, left site, first operand on the left) | ("swap", k) | ("pswap", k, prod_left) |
    ("read", name, site, aux).  With return_layout, also pos (logical qubit -> final site)."""
    resets = [[] for _ in range(n)]
    gates2 = [[] for _ in range(n)]
    for i, (name, qs, _) in enumerate(ops):
        if name == "R":
            resets[qs[0]].append(i)
        elif name in ("CX", "CZ", "SWAP"):
            gates2[qs[0]].append(i)
            gates2[qs[1]].append(i)

    def nxt(v, i):
        j = bisect.bisect_right(v, i)
        return v[j] if j < len(v) else -1

    pos, at, prod = list(range(n)), list(range(n)), [True] * n
    steps = []

    def swap(k):
        x, y = at[k], at[k + 1]
        steps.append(("pswap", k, prod[x]) if (prod[x] or prod[y]) else ("swap", k))
        at[k], at[k + 1] = y, x
        pos[x], pos[y] = k + 1, k

    for i, (name, qs, aux) in enumerate(ops):
        if name in ("DEP1", "DEP2", "XERR"):
            steps.append(("ch", name, tuple(pos[q] for q in qs), aux))
        elif name == "SWAP":
            a, b = qs
            pos[a], pos[b] = pos[b], pos[a]
            at[pos[a]], at[pos[b]] = a, b
            prod[a], prod[b] = prod[b], prod[a]
        elif name in ("CX", "CZ"):
            a, b = qs
            if prod[a] != prod[b]:
                mv = a if prod[a] else b
            else:
                ra, rb = nxt(resets[a], i), nxt(resets[b], i)
                if ra != rb and (ra >= 0 or rb >= 0):
                    mv = a if (rb < 0 or (0 <= ra < rb)) else b
                else:
                    def score(m_, o_):
                        d = abs(pos[m_] - pos[o_]) - 1
                        dest = pos[o_] - 1 if pos[m_] < pos[o_] else pos[o_] + 1
                        j = nxt(gates2[m_], i)
                        if j >= 0:
                            q2 = ops[j][1]
                            partner = q2[1] if q2[0] == m_ else q2[0]
                            if partner != o_:
                                d += 0.5 * max(0, abs(dest - pos[partner]) - 1)
                        return d
                    mv = a if score(a, b) <= score(b, a) else b
            other = b if mv == a else a
            while abs(pos[mv] - pos[other]) > 1:
                swap(pos[mv] if pos[mv] < pos[other] else pos[mv] - 1)
            steps.append(("g2", name, min(pos[a], pos[b]), pos[a] < pos[b]))
            prod[a] = prod[b] = False
        elif name in ("M", "R"):
            q = qs[0]
            steps.append(("read", name, pos[q], aux))
            prod[q] = True
            if name == "R":
                while pos[q] != q:
                    swap(pos[q] - 1 if pos[q] > q else pos[q])
        else:
            steps.append(("1q", name, pos[qs[0]]))
    return (steps, pos) if return_layout else steps


def n_svd_updates(steps):
    return sum(1 for st in steps if st[0] in ("g2", "swap"))


def run_shot(n, ops, faults, *, seed, shot, chi_max, cutoff, dev, max_updates=None, steps=None):
    """One shot; returns (status, updates).  faults: dict channel -> pauli code."""
    one, two, paulis = _gates(dev)
    m = PlainMPS(n, chi_max, cutoff, dev)
    sw = two["SWAP"]
    for st in (steps if steps is not None else plan(n, ops)):
        if max_updates is not None and m.updates >= max_updates:
            return "cut", m.updates
        kind = st[0]
        if kind == "1q":
            m.one(one[st[1]], st[2])
        elif kind == "g2":
            g = two[st[1]]
            m.two_site(g if st[3] else sw @ g @ sw, st[2])
        elif kind == "swap":
            m.two_site(sw, st[1])
        elif kind == "pswap":
            m.product_swap(st[1], st[2])
        elif kind == "ch":
            code = faults.get(st[3])
            if code:
                if st[1] == "DEP2":
                    m.one(paulis[code >> 2], st[2][0])
                    m.one(paulis[code & 3], st[2][1])
                else:
                    m.one(paulis[code], st[2][0])
        else:
            q = st[2]
            p1 = m.prob1(q)
            o = 1 if readout_uniform(seed, st[3], shot) < p1 else 0
            if st[1] == "M" and o == 1:
                return "rejected", m.updates
            m.project(q, o)
            if st[1] == "R" and o == 1:
                m.one(one["X"], q)
    if str(dev).startswith("cuda"):
        torch.cuda.synchronize()
    return "accepted", m.updates
