"""Gate matrices and Pauli codes for the oracle (test infrastructure only).

Conventions: a two-qubit gate on (a, b) is a 4x4 matrix over |q_a q_b> with q_a the high bit.
CX(c, t) flips t when c is 1.  T = diag(1, e^{i pi/4}) (Sec. 1: |T> = T|+>).
"""
from __future__ import annotations

import numpy as np

SQ2 = np.sqrt(0.5)
I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
H = np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=complex)
S = np.diag([1, 1j]).astype(complex)
SDG = np.diag([1, -1j]).astype(complex)
T = np.diag([1, np.exp(1j * np.pi / 4)]).astype(complex)
TDG = np.diag([1, np.exp(-1j * np.pi / 4)]).astype(complex)
ONE_Q = {"H": H, "S": S, "SDG": SDG, "X": X, "Y": Y, "Z": Z, "T": T, "TDG": TDG}

CX = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
CZ = np.diag([1, 1, 1, -1]).astype(complex)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
TWO_Q = {"CX": CX, "CZ": CZ, "SWAP": SWAP}

PAULI = [I2, X, Y, Z]  # index 0=I 1=X 2=Y 3=Z


def fault_paulis(kind: str, code: int):
    """The Pauli factors of a fault: one factor for DEP1/XERR, two for DEP2 (Sec. 4, 4^k-1)."""
    if kind == "DEP2":
        return [PAULI[code >> 2], PAULI[code & 3]]
    return [PAULI[code]]
