"""FP64 matrix-product-state simulation of one shot (Sec. 3.1, Eq. 1), test infrastructure only.

A state of n qubits on a line is a chain of site tensors A[k] with index order (left bond,
physical, right bond) (Eq. 1).  Bond k sits between sites k and k+1; its dimension is the number
of kept singular values of the split across that cut (Sec. 3.1).  The chain is kept in mixed
canonical form with a single orthogonality centre, moved by QR steps.

Two-site update on adjacent sites (q, q+1): move the centre to q, contract
theta[(l,s),(t,r)] = sum_m A[q][l,s,m] A[q+1][m,t,r], apply the 4x4 gate on the physical pair,
SVD theta, keep r values by the truncation rule below, A[q] = U, A[q+1] = S V^dagger (centre on
q+1).  A gate between sites at line distance d > 1 is routed with SWAPs (Sec. 3.1: its cost
grows with the distance on the chain): SWAP on (lo+i, lo+i+1) for i = 0..d-2, the gate on
(hi-1, hi), then the same SWAPs in reverse order; every SWAP is itself a two-site update.

Truncation rule (the paper runs without truncation, Sec. 5.1; the kept count is otherwise not
fixed by it): singular values sorted descending; r is the smallest count >= 1 whose discarded
tail sum_{i>=r} s_i^2 is <= cutoff * sum_i s_i^2, then r = min(r, chi_max).  The kept values are
rescaled so that their squares sum to 1, and the discarded fraction of sum s^2 is added to the
shot's discarded weight.  A cut is flagged degenerate when the last kept and first discarded
singular values agree to a relative 1e-8 (the kept subspace is then not unique).
"""
from __future__ import annotations

import numpy as np

from . import gates
from .philox import readout_uniform
from .statevector import REF_RESET_THRESHOLD


class MPS:
    def __init__(self, n: int, chi_max: int = 1 << 30, cutoff: float = 0.0):
        self.n = n
        self.chi_max = chi_max
        self.cutoff = cutoff
        self.A = [np.zeros((1, 2, 1), dtype=np.complex128) for _ in range(n)]
        for a in self.A:
            a[0, 0, 0] = 1.0
        self.center = 0
        self.discarded = 0.0
        self.degenerate_cuts = 0
        self.chi_peak = 1
        self.updates = 0

    def bond_dims(self):
        return [self.A[k].shape[2] for k in range(self.n - 1)]

    # -- canonical centre --------------------------------------------------------------------
    def _shift_right(self, q):
        a = self.A[q]
        l, d, r = a.shape
        qm, rm = np.linalg.qr(a.reshape(l * d, r))
        self.A[q] = qm.reshape(l, d, qm.shape[1])
        self.A[q + 1] = np.tensordot(rm, self.A[q + 1], axes=([1], [0]))

    def _shift_left(self, q):
        a = self.A[q]
        l, d, r = a.shape
        qm, rm = np.linalg.qr(a.reshape(l, d * r).conj().T)
        self.A[q] = qm.conj().T.reshape(qm.shape[1], d, r)
        self.A[q - 1] = np.tensordot(self.A[q - 1], rm.conj().T, axes=([2], [0]))

    def move_center(self, q):
        while self.center < q:
            self._shift_right(self.center)
            self.center += 1
        while self.center > q:
            self._shift_left(self.center)
            self.center -= 1

    # -- gates -------------------------------------------------------------------------------
    def apply1(self, u, q):
        self.A[q] = np.einsum("st,ltr->lsr", u, self.A[q])

    def _truncate(self, s):
        s2 = s.astype(np.float64) ** 2
        tot = float(np.sum(s2))
        tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[r] = sum_{i>=r} s_i^2
        r = 1
        while r < len(s) and tail[r] > self.cutoff * tot:
            r += 1
        r = min(r, self.chi_max)
        if r < len(s) and s[r] > 0 and s[r - 1] / s[r] - 1.0 < 1e-8:
            self.degenerate_cuts += 1
        self.discarded += float(tail[r] / tot) if tot > 0 else 0.0
        return r

    def apply2_adjacent(self, u4, q):
        """Gate u4 on (q, q+1) with qubit q as the high bit of the 4x4 index."""
        self.move_center(q)
        a, b = self.A[q], self.A[q + 1]
        l, r = a.shape[0], b.shape[2]
        theta = np.einsum("lsm,mtr->lstr", a, b)
        theta = np.einsum("stuv,luvr->lstr", u4.reshape(2, 2, 2, 2), theta)
        um, s, vh = np.linalg.svd(theta.reshape(2 * l, 2 * r), full_matrices=False)
        k = self._truncate(s)
        sk = s[:k] / np.sqrt(np.sum(s[:k].astype(np.float64) ** 2))
        self.A[q] = um[:, :k].reshape(l, 2, k)
        self.A[q + 1] = (sk[:, None] * vh[:k]).reshape(k, 2, r)
        self.center = q + 1
        self.chi_peak = max(self.chi_peak, k)
        self.updates += 1

    def apply2(self, u4, a, b):
        """Gate u4 on qubits (a, b) (a is the high bit), routed with SWAPs when not adjacent."""
        if abs(a - b) == 1:
            if a < b:
                self.apply2_adjacent(u4, a)
            else:
                sw = gates.SWAP
                self.apply2_adjacent(sw @ u4 @ sw, b)
            return
        lo, hi = min(a, b), max(a, b)
        for i in range(lo, hi - 1):
            self.apply2_adjacent(gates.SWAP, i)
        # the qubit from lo now sits at hi-1
        if a < b:
            self.apply2_adjacent(u4, hi - 1)
        else:
            sw = gates.SWAP
            self.apply2_adjacent(sw @ u4 @ sw, hi - 1)
        for i in range(hi - 2, lo - 1, -1):
            self.apply2_adjacent(gates.SWAP, i)

    # -- readout -----------------------------------------------------------------------------
    def prob1(self, q) -> float:
        self.move_center(q)
        a = self.A[q]
        p0 = float(np.sum(np.abs(a[:, 0, :]) ** 2))
        p1 = float(np.sum(np.abs(a[:, 1, :]) ** 2))
        return p1 / (p0 + p1)

    def project(self, q, outcome):
        self.move_center(q)
        a = self.A[q].copy()
        a[:, 1 - outcome, :] = 0.0
        a /= np.sqrt(np.sum(np.abs(a) ** 2))
        self.A[q] = a

    def vector(self):
        """Dense state (small n only), qubit 0 as the highest bit."""
        v = self.A[0]
        for k in range(1, self.n):
            v = np.tensordot(v, self.A[k], axes=([-1], [0]))
        return v.reshape(-1)

    def norm2(self) -> float:
        return float(np.real(overlap(self, self)))


def overlap(a: MPS, b: MPS) -> complex:
    """<a|b> by a left-to-right transfer-matrix sweep, O(n chi^3)."""
    e = np.ones((1, 1), dtype=np.complex128)
    for k in range(a.n):
        # e[i, j] over (bond of a, bond of b)
        t = np.tensordot(e, b.A[k], axes=([1], [0]))                     # (ia, s, rb)
        e = np.tensordot(a.A[k].conj(), t, axes=([0, 1], [0, 1]))        # (ra, rb)
    return complex(e[0, 0])


def fidelity(a: MPS, b: MPS) -> float:
    ov = overlap(a, b)
    return float(abs(ov) ** 2 / (overlap(a, a).real * overlap(b, b).real))


def run_shot(circ, faults=(), *, seed=0, shot=0, chi_max=1 << 30, cutoff=0.0, reference=False,
             record=None):
    """One shot on the MPS; same semantics and readout draws as statevector.run_shot."""
    m = MPS(circ.n, chi_max, cutoff)
    fmap = {} if reference else dict(faults)
    for idx, (name, qs) in enumerate(circ.ops):
        if name in gates.ONE_Q:
            m.apply1(gates.ONE_Q[name], qs[0])
        elif name in gates.TWO_Q:
            m.apply2(gates.TWO_Q[name], qs[0], qs[1])
        elif name in ("DEP1", "DEP2", "XERR"):
            c = circ.channel_of_op[idx]
            if c in fmap:
                for q, pm in zip(qs, gates.fault_paulis(name, fmap[c])):
                    m.apply1(pm, q)
        elif name in ("M", "R"):
            q = qs[0]
            p1 = m.prob1(q)
            if record is not None:
                record.append((idx, p1))
            if reference:
                if name == "M":
                    if p1 > 1e-10:
                        raise ValueError(f"measurement at op {idx} is not deterministic in the noiseless circuit")
                    outcome = 0
                else:
                    outcome = 1 if p1 > REF_RESET_THRESHOLD else 0
            else:
                u = readout_uniform(seed, circ.readout_of_op[idx], shot)
                outcome = 1 if u < p1 else 0
            if name == "M" and outcome == 1:
                return "rejected", m, idx
            m.project(q, outcome)
            if name == "R" and outcome == 1:
                m.apply1(gates.X, q)
        else:
            raise ValueError(name)
    return "accepted", m, None
