"""Seeded random Clifford+T circuits (unstructured) in the qcmps circuit text format.

Used to exercise every gate, every line distance and non-deterministic measurements; these
circuits do not have the cultivation shape.  Only input construction lives here.
"""
from __future__ import annotations

import numpy as np

ONE_Q = ("H", "S", "SDG", "X", "Y", "Z", "T", "TDG")
TWO_Q = ("CX", "CZ", "SWAP")


def random_circuit(n: int, n_ops: int, *, seed: int = 0, max_dist: int = 3, p_meas: float = 0.0,
                   p_reset: float = 0.0, noise: bool = True, clifford_only: bool = False,
                   one_q=None, two_q=None) -> str:
    rng = np.random.default_rng(np.random.PCG64([seed, n, n_ops, 7]))
    one_q = tuple(one_q) if one_q is not None else (
        tuple(g for g in ONE_Q if g not in ("T", "TDG")) if clifford_only else ONE_Q)
    two_q = tuple(two_q) if two_q is not None else TWO_Q
    out = [f"# random circuit n={n} ops={n_ops} seed={seed}", f"QUBITS {n}"]
    for _ in range(n_ops):
        u = rng.random()
        if u < p_meas:
            q = int(rng.integers(n))
            if noise:
                out.append(f"XERR {q}")
            out.append(f"M {q}")
        elif u < p_meas + p_reset:
            q = int(rng.integers(n))
            out.append(f"R {q}")
            if noise:
                out.append(f"XERR {q}")
        elif n >= 2 and rng.random() < 0.5:
            a = int(rng.integers(n))
            lo, hi = max(0, a - max_dist), min(n - 1, a + max_dist)
            b = a
            while b == a:
                b = int(rng.integers(lo, hi + 1))
            g = two_q[int(rng.integers(len(two_q)))]
            out.append(f"{g} {a} {b}")
            if noise:
                out.append(f"DEP2 {a} {b}")
        else:
            q = int(rng.integers(n))
            g = one_q[int(rng.integers(len(one_q)))]
            out.append(f"{g} {q}")
            if noise:
                out.append(f"DEP1 {q}")
    return "\n".join(out) + "\n"
