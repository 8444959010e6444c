"""FP64 state-vector simulation of one shot: the plain definition of what is sampled (Sec. 4).

Test infrastructure only.  A shot applies the circuit with its fault configuration inserted as
Pauli gates; each Z measurement draws its outcome from the Born rule and the shot is discarded at
the first measurement that returns 1 (Sec. 4 and App. A.3: every measurement is post-selected on
0).  An accepted shot is compared with the noiseless reference state: a logical error is flagged
when the normalised squared overlap differs from 1 (Sec. 4 and App. A.3; the synthetic circuits
have no decoder, so the reference is the noiseless final state itself).
"""
from __future__ import annotations

import numpy as np

from . import gates
from .philox import readout_uniform

MAX_QUBITS = 26

# Reference run: a reset of a qubit that is not in a definite state takes outcome 1 only when
# p1 exceeds this value.  The paper's reference is the noiseless final state (App. A.3); its
# resets follow post-selected measurements and are deterministic.  For other circuits a fixed
# convention is needed, and a threshold away from the values Clifford+T amplitudes produce
# (1/2, cos^2(pi/8), ...) keeps the choice immune to rounding.
REF_RESET_THRESHOLD = 0.6180339887498949


class StateVector:
    def __init__(self, n: int):
        if n > MAX_QUBITS:
            raise ValueError("too many qubits for the state-vector oracle")
        self.n = n
        self.psi = np.zeros((2,) * n, dtype=np.complex128)
        self.psi[(0,) * n] = 1.0

    def apply1(self, u, q):
        """psi[..., s, ...] <- sum_t u[s, t] psi[..., t, ...] on axis q."""
        v = self.psi.reshape(2 ** q, 2, 2 ** (self.n - q - 1))
        self.psi = np.einsum("st,ltr->lsr", u, v).reshape((2,) * self.n)

    def apply2(self, u4, a, b):
        """4x4 gate on axes (a, b), a being the high bit of the gate index."""
        g = u4.reshape(2, 2, 2, 2)
        out = np.tensordot(g, self.psi, axes=([2, 3], [a, b]))
        self.psi = np.moveaxis(out, [0, 1], [a, b])

    def prob1(self, q) -> float:
        """Born probability of outcome 1 on qubit q, normalised by the state norm."""
        sl = [slice(None)] * self.n
        sl[q] = 1
        p1 = float(np.sum(np.abs(self.psi[tuple(sl)]) ** 2))
        tot = float(np.sum(np.abs(self.psi) ** 2))
        return p1 / tot

    def project(self, q, outcome):
        sl = [slice(None)] * self.n
        sl[q] = 1 - outcome
        self.psi[tuple(sl)] = 0.0
        self.psi /= np.sqrt(np.sum(np.abs(self.psi) ** 2))

    def vector(self):
        return self.psi.reshape(-1)


def apply_op(sv, name, qs):
    if name in gates.ONE_Q:
        sv.apply1(gates.ONE_Q[name], qs[0])
    elif name in gates.TWO_Q:
        sv.apply2(gates.TWO_Q[name], qs[0], qs[1])
    else:
        raise ValueError(name)


def run_shot(circ, faults=(), *, seed=0, shot=0, reference=False, record=None):
    """Run one shot.  faults: sorted (channel, code) pairs.  Returns (status, state, probs).

    status is 'rejected' at the first measurement returning 1, else 'accepted'.  With
    reference=True no faults are applied, every measurement is projected on 0 and a reset takes
    outcome 1 only when p1 > REF_RESET_THRESHOLD; a measurement with p1 > 1e-10 then raises (the noiseless
    circuit must return 0 deterministically for the overlap test to be defined).
    record: optional list receiving (op index, p1) for every readout."""
    sv = StateVector(circ.n)
    fmap = {} if reference else dict(faults)
    for idx, (name, qs) in enumerate(circ.ops):
        if name in gates.ONE_Q or name in gates.TWO_Q:
            apply_op(sv, name, qs)
        elif name in ("DEP1", "DEP2", "XERR"):
            c = circ.channel_of_op[idx]
            if c in fmap:
                for q, pm in zip(qs, gates.fault_paulis(name, fmap[c])):
                    sv.apply1(pm, q)
        elif name in ("M", "R"):
            q = qs[0]
            p1 = sv.prob1(q)
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
                return "rejected", sv, idx
            sv.project(q, outcome)
            if name == "R" and outcome == 1:
                sv.apply1(gates.X, q)
        else:
            raise ValueError(name)
    return "accepted", sv, None


def fidelity(a, b) -> float:
    """Normalised squared overlap |<a|b>|^2 / (<a|a><b|b>)."""
    va, vb = a.vector(), b.vector()
    ov = np.vdot(va, vb)
    return float(abs(ov) ** 2 / (np.vdot(va, va).real * np.vdot(vb, vb).real))
