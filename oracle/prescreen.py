"""Offline screening and the per-shot Pauli pre-screen (Sec. 4.2), test infrastructure only.

Offline analysis (Sec. 4.2): starting from the stabilisers +Z_i of |0...0>, track the stabiliser
group through the circuit.  Clifford gates conjugate it.  The non-Clifford gates are diagonal
(T, T^dagger here), so a group element with I or Z on their support passes through unchanged;
the elements that do not commute are dropped, keeping the largest subgroup with no X component
on the support (Gaussian elimination first, so the result does not depend on the generator
basis).  At a Z measurement the outcome is decided when +-Z_q belongs to the tracked group.  After
a measurement (post-selected on 0) or a reset, the anticommuting part is dropped and +Z_q added.
Only shapes (X/Z bit patterns) are tracked: Pauli noise changes signs, never shapes (Sec. 4.2).

Per-shot pre-screen (Sec. 4.2): a Pauli frame (x_q, z_q) per qubit starts at 0; a fault XORs its
Pauli into the frame; Clifford gates conjugate the frame; diagonal non-Clifford gates leave it
alone; a measurement's flip is x_q, after which the qubit's frame is cleared (as at a reset).  The
shot is discarded when any decided measurement flips.  This is unbiased: it only removes shots
that post-selection would reject with certainty (Sec. 4.2).

The paper precompiles the effect of each noise channel on the measurements over GF(2) (Sec. 4.2,
following SymFT); `sensitivity_matrix` is that second route, computed by propagating every
decided measurement's Z_q backwards, and must agree with the frame bit for bit.
"""
from __future__ import annotations

import numpy as np

CLIFFORD1 = {"H", "S", "SDG", "X", "Y", "Z"}
DIAGONAL_NON_CLIFFORD = {"T", "TDG"}


def _conj_shape(x, z, name, qs):
    """Conjugate Pauli shapes (rows of x, z bit arrays) by a Clifford gate, in place.

    The shape map of each of these gates is its own inverse, so the same update serves forward
    (frame) and backward (Heisenberg) propagation."""
    if name == "H":
        a = qs[0]
        x[..., a], z[..., a] = z[..., a].copy(), x[..., a].copy()
    elif name in ("S", "SDG"):
        a = qs[0]
        z[..., a] ^= x[..., a]
    elif name == "CX":
        c, t = qs
        x[..., t] ^= x[..., c]
        z[..., c] ^= z[..., t]
    elif name == "CZ":
        a, b = qs
        z[..., a] ^= x[..., b]
        z[..., b] ^= x[..., a]
    elif name == "SWAP":
        a, b = qs
        x[..., a], x[..., b] = x[..., b].copy(), x[..., a].copy()
        z[..., a], z[..., b] = z[..., b].copy(), z[..., a].copy()
    elif name in ("X", "Y", "Z"):
        pass
    else:
        raise ValueError(name)


def _rank(m):
    m = m.copy()
    rank = 0
    rows, cols = m.shape
    for c in range(cols):
        piv = np.nonzero(m[rank:, c])[0]
        if len(piv) == 0:
            continue
        p = rank + piv[0]
        m[[rank, p]] = m[[p, rank]]
        for r in range(rows):
            if r != rank and m[r, c]:
                m[r] ^= m[rank]
        rank += 1
        if rank == rows:
            break
    return rank


class StabiliserGroup:
    """Generators of the tracked group as shape rows [x | z] (uint8)."""

    def __init__(self, n):
        self.n = n
        self.x = np.zeros((n, n), dtype=np.uint8)
        self.z = np.eye(n, dtype=np.uint8)

    def conj(self, name, qs):
        _conj_shape(self.x, self.z, name, qs)

    def drop_x_on(self, q):
        """Keep the subgroup of elements with no X component on qubit q."""
        rows = np.nonzero(self.x[:, q])[0]
        if len(rows) == 0:
            return
        p = rows[0]
        for r in rows[1:]:
            self.x[r] ^= self.x[p]
            self.z[r] ^= self.z[p]
        self.x = np.delete(self.x, p, axis=0)
        self.z = np.delete(self.z, p, axis=0)

    def contains_z(self, q) -> bool:
        m = np.concatenate([self.x, self.z], axis=1)
        v = np.zeros((1, 2 * self.n), dtype=np.uint8)
        v[0, self.n + q] = 1
        return _rank(np.concatenate([m, v])) == _rank(m)

    def add_z(self, q):
        if self.contains_z(q):
            return
        zr = np.zeros((1, self.n), dtype=np.uint8)
        zr[0, q] = 1
        self.x = np.concatenate([self.x, np.zeros((1, self.n), dtype=np.uint8)])
        self.z = np.concatenate([self.z, zr])


def decided_measurements(circ):
    """Per op index of every M: True when stabiliser tracking decides its outcome (Sec. 4.2)."""
    g = StabiliserGroup(circ.n)
    decided = {}
    for idx, (name, qs) in enumerate(circ.ops):
        if name in CLIFFORD1 or name in ("CX", "CZ", "SWAP"):
            g.conj(name, qs)
        elif name in DIAGONAL_NON_CLIFFORD:
            g.drop_x_on(qs[0])
        elif name == "M":
            decided[idx] = g.contains_z(qs[0])
            g.drop_x_on(qs[0])
            g.add_z(qs[0])
        elif name == "R":
            g.drop_x_on(qs[0])
            g.add_z(qs[0])
        elif name in ("DEP1", "DEP2", "XERR"):
            pass
        else:
            raise ValueError(name)
    return decided


_PAULI_XZ = {0: (0, 0), 1: (1, 0), 2: (1, 1), 3: (0, 1)}


def _fault_xz(kind, code):
    if kind == "DEP2":
        return [_PAULI_XZ[code >> 2], _PAULI_XZ[code & 3]]
    return [_PAULI_XZ[code]]


def frame_prescreen(circ, decided, faults_by_shot):
    """Kept flag per shot by forward Pauli-frame propagation (Sec. 4.2), vectorised over shots.

    faults_by_shot: dict shot -> sorted list of (channel, code)."""
    shots = list(faults_by_shot)
    S = len(shots)
    x = np.zeros((S, circ.n), dtype=np.uint8)
    z = np.zeros((S, circ.n), dtype=np.uint8)
    rejected = np.zeros(S, dtype=bool)
    # faults indexed by channel: list of (shot row, code)
    by_channel = {}
    for row, s in enumerate(shots):
        for c, code in faults_by_shot[s]:
            by_channel.setdefault(c, []).append((row, code))
    for idx, (name, qs) in enumerate(circ.ops):
        if name in CLIFFORD1 or name in ("CX", "CZ", "SWAP"):
            _conj_shape(x, z, name, qs)
        elif name in DIAGONAL_NON_CLIFFORD:
            pass
        elif name in ("DEP1", "DEP2", "XERR"):
            c = circ.channel_of_op[idx]
            for row, code in by_channel.get(c, ()):
                for q, (px, pz) in zip(qs, _fault_xz(name, code)):
                    x[row, q] ^= px
                    z[row, q] ^= pz
        elif name == "M":
            q = qs[0]
            if decided[idx]:
                rejected |= x[:, q].astype(bool)
            x[:, q] = 0
            z[:, q] = 0
        elif name == "R":
            x[:, qs[0]] = 0
            z[:, qs[0]] = 0
        else:
            raise ValueError(name)
    return {s: not bool(rejected[row]) for row, s in enumerate(shots)}


def sensitivity_matrix(circ, decided):
    """GF(2) matrix sens[channel][code] -> bit vector over decided measurements (Sec. 4.2).

    Each decided measurement's Z_q is propagated backwards through the Clifford skeleton (diagonal
    non-Cliffords as identity); at an earlier measurement or reset of qubit r the operator loses its
    component on r (the reset fixes Z_r = +1 regardless of what came before).  A fault flips the
    measurement iff it anticommutes with the propagated operator at its own position."""
    dec_ops = [i for i, (nm, _) in enumerate(circ.ops) if nm == "M" and decided[i]]
    D = len(dec_ops)
    col_of = {op: j for j, op in enumerate(dec_ops)}
    x = np.zeros((D, circ.n), dtype=np.uint8)  # row j = operator of decided measurement j
    z = np.zeros((D, circ.n), dtype=np.uint8)
    sens = {}
    for idx in range(len(circ.ops) - 1, -1, -1):
        name, qs = circ.ops[idx]
        if name in CLIFFORD1 or name in ("CX", "CZ", "SWAP"):
            _conj_shape(x, z, name, qs)
        elif name in DIAGONAL_NON_CLIFFORD:
            pass
        elif name in ("DEP1", "DEP2", "XERR"):
            c = circ.channel_of_op[idx]
            codes = [1] if name == "XERR" else (range(1, 16) if name == "DEP2" else range(1, 4))
            rows = {}
            for code in codes:
                bits = np.zeros(D, dtype=np.uint8)
                for q, (px, pz) in zip(qs, _fault_xz(name, code)):
                    bits ^= (px & z[:, q]) ^ (pz & x[:, q])
                rows[code] = bits
            sens[c] = rows
        elif name in ("M", "R"):
            q = qs[0]
            x[:, q] = 0
            z[:, q] = 0
            if name == "M" and idx in col_of:
                z[col_of[idx], q] = 1
        else:
            raise ValueError(name)
    return sens, dec_ops


def gf2_prescreen(circ, decided, faults_by_shot):
    """Kept flag per shot from the sensitivity matrix: XOR of the faults' rows."""
    sens, dec_ops = sensitivity_matrix(circ, decided)
    out = {}
    for s, faults in faults_by_shot.items():
        v = np.zeros(len(dec_ops), dtype=np.uint8)
        for c, code in faults:
            v ^= sens[c][code]
        out[s] = not bool(v.any())
    return out
