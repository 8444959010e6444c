"""Seeded synthetic cultivation-shaped Clifford+T circuits in the qcmps circuit text format.

The paper's own cultivation circuits (Sec. 2, App. A.1) are not available, so the workloads are
synthetic stand-ins with their shape: a line of qubits with data at even and ancillas at odd
positions (17 = 9 + 8 for the d=3 shape, 49 = 25 + 24 for the d=5 shape), a unitary encoding
stage, then check layers whose every ancilla measurement is post-selected on 0 (Sec. 4, App. A.3),
with T gates spread over data and ancilla qubits and uniform depolarising noise after every
gate and X errors before measurements and after resets (Sec. 4 and App. A.2).

One layer is built so that every ancilla returns to |0> in the noiseless circuit (each check is
an echo that undoes itself), while the data register carries a state whose entanglement stays
bounded, as the paper's cultivation states do (Table 1: chi_peak 8-96, exact MPS):

  1. frame   V: H or S on every data qubit, then random disjoint CNOTs between neighbouring data
             qubits (line distance 2);
  2. open    every ancilla a couples to two data partners at line distance 1 or 3, either as a
             Z echo  CX(d1->a) CX(d2->a)                       (decided by stabiliser tracking),
             or, where a T placement hits the ancilla, as a
             magic echo H(a) T(a) CZ(a,d1) CZ(a,d2)            (undecided: needs the simulator);
  3. window  T on the data qubits that this layer's T placements hit;
  4. close   the openings in reverse order (magic echoes end with T^dagger(a), H(a));
  5. frame   V^dagger;
  6. readout X error, M, R, X error on every ancilla.

The text format is one instruction per line:  QUBITS n | H q | S q | SDG q | X q | Y q | Z q |
T q | TDG q | CX c t | CZ a b | SWAP a b | M q | R q | DEP1 q | DEP2 a b | XERR q | TICK, with
'#' comments.  Every M is a Z-basis measurement post-selected on outcome 0.  Noise instructions
carry no rate: the rate p is uniform over all channels and is a parameter of the sampling call.

This module only builds inputs; it holds none of the simulation arithmetic.
"""
from __future__ import annotations

import numpy as np

__all__ = ["cultivation_circuit", "WORKLOADS", "workload_circuit", "tiny_circuit"]


def _t_placements(rng, n, layers, t_per_layer, t_total):
    placed = set()
    if t_per_layer is not None:
        for layer in range(layers):
            for q in rng.choice(n, size=min(t_per_layer, n), replace=False):
                placed.add((layer, int(q)))
    if t_total is not None:
        cells = rng.choice(layers * n, size=min(t_total, layers * n), replace=False)
        for cell in cells:
            placed.add((int(cell) // n, int(cell) % n))
    return placed


def cultivation_circuit(n_data: int, layers: int, *, seed: int = 0, t_per_layer: int | None = None,
                        t_total: int | None = None, enc_rounds: int = 4, enc_density: float = 0.75, enc_mix: float = 0.5,
                        data_cx_prob: float = 0.5, far_prob: float = 0.5, noise: bool = True,
                        prefix_layers: int | None = None) -> str:
    """Return the circuit text of a seeded cultivation-shaped circuit.

    n_data       data qubits (the line has 2*n_data-1 qubits)
    layers       check layers, each ending with measure-and-reset of every ancilla
    t_per_layer  T placements drawn per layer (d=3 shape: 4), or
    t_total      T placements drawn over the whole circuit (d=5 shape: 16)
    enc_rounds   brickwork rounds of the encoding stage (bounds the data entanglement)
    enc_density  probability of a CNOT on each brickwork pair
    enc_mix      probability of an H or S on each data qubit after each brickwork round
    prefix_layers  emit only the first prefix_layers check layers of this circuit (all random draws
                 are made as for the full circuit, so the result is a true prefix of it)
    """
    if n_data < 2:
        raise ValueError("need at least two data qubits")
    rng = np.random.default_rng(np.random.PCG64([seed, n_data, layers]))
    n = 2 * n_data - 1
    data = [2 * i for i in range(n_data)]
    anc = [2 * i + 1 for i in range(n_data - 1)]
    out = [f"# cultivation-shaped synthetic circuit: n_data={n_data} layers={layers} seed={seed}",
           f"QUBITS {n}"]

    def g1(name, q):
        out.append(f"{name} {q}")
        if noise:
            out.append(f"DEP1 {q}")

    def g2(name, a, b):
        out.append(f"{name} {a} {b}")
        if noise:
            out.append(f"DEP2 {a} {b}")

    # Encoding: random H layer, then brickwork CNOT rounds between neighbouring data qubits.
    out.append("# encoding")
    for q in data:
        if rng.random() < 0.5:
            g1("H", q)
    for r in range(enc_rounds):
        for i in range(r % 2, n_data - 1, 2):
            if rng.random() < enc_density:
                c, t = (data[i], data[i + 1]) if rng.random() < 0.5 else (data[i + 1], data[i])
                g2("CX", c, t)
        for q in data:
            u = rng.random()
            if u < enc_mix / 2:
                g1("H", q)
            elif u < enc_mix:
                g1("S", q)

    placed = _t_placements(rng, n, layers, t_per_layer, t_total)

    emit = layers if prefix_layers is None else max(0, min(layers, prefix_layers))
    for layer in range(layers):
        if layer == emit:  # the remaining layers are drawn (same random sequence) but not emitted
            keep = len(out)
        out.append("TICK")
        out.append(f"# layer {layer}")
        frame = ["H" if rng.random() < 0.5 else "S" for _ in data]
        for q, g in zip(data, frame):
            g1(g, q)
        pairs = []
        i = 0
        while i < n_data - 1:
            if rng.random() < data_cx_prob:
                pairs.append((data[i], data[i + 1]) if rng.random() < 0.5 else (data[i + 1], data[i]))
                i += 2
            else:
                i += 1
        for c, t in pairs:
            g2("CX", c, t)
        checks = []
        for ai, a in enumerate(anc):
            d1 = data[ai - 1] if (ai - 1 >= 0 and rng.random() < far_prob) else data[ai]
            d2 = data[ai + 2] if (ai + 2 < n_data and rng.random() < far_prob) else data[ai + 1]
            checks.append((a, d1, d2, (layer, a) in placed))
        for a, d1, d2, magic in checks:
            if magic:
                g1("H", a)
                g1("T", a)
                g2("CZ", a, d1)
                g2("CZ", a, d2)
            else:
                g2("CX", d1, a)
                g2("CX", d2, a)
        for q in data:
            if (layer, q) in placed:
                g1("T", q)
        for a, d1, d2, magic in reversed(checks):
            if magic:
                g2("CZ", a, d2)
                g2("CZ", a, d1)
                g1("TDG", a)
                g1("H", a)
            else:
                g2("CX", d2, a)
                g2("CX", d1, a)
        for c, t in reversed(pairs):
            g2("CX", c, t)
        for q, g in zip(data, frame):
            g1("H" if g == "H" else "SDG", q)
        for a in anc:
            if noise:
                out.append(f"XERR {a}")
            out.append(f"M {a}")
            out.append(f"R {a}")
            if noise:
                out.append(f"XERR {a}")
    if emit < layers:
        out = out[:keep]
    return "\n".join(out) + "\n"


# The workloads, named by shape and size.
WORKLOADS = {
    # 17 qubits (9 data + 8 ancilla), 12 layers, 4 T per layer; noiseless chi_peak 16
    "d3_17q_12l": dict(n_data=9, layers=12, t_per_layer=4, enc_rounds=4, enc_density=1.0, enc_mix=1.0),
    # 49 qubits (25 data + 24 ancilla), 200 layers, 16 T in total: pre-screen workload
    "d5_49q_200l": dict(n_data=25, layers=200, t_total=16, enc_rounds=12, enc_density=1.0, enc_mix=1.0),
    # 49 qubits (25 data + 24 ancilla), 60 layers, 16 T in total: batched MPS workload;
    # noiseless chi_peak 64
    "d5_49q_60l": dict(n_data=25, layers=60, t_total=16, enc_rounds=12, enc_density=1.0, enc_mix=1.0),
    # the same shape with a deeper encoding, so that the data register carries more entanglement:
    # the encoded stabiliser state has bond 64 at the middle and the check layers reach bond 128
    # (24 rounds) or 256 (28 rounds), all exact at chi_max 256
    "d5_49q_60l_b128": dict(n_data=25, layers=60, t_total=16, enc_rounds=24, enc_density=1.0, enc_mix=1.0),
    "d5_49q_60l_b256": dict(n_data=25, layers=60, t_total=16, enc_rounds=28, enc_density=1.0, enc_mix=1.0),
}


def workload_circuit(name: str, seed: int = 0, **overrides) -> str:
    kw = dict(WORKLOADS[name])
    kw.update(overrides)
    return cultivation_circuit(seed=seed, **kw)


def tiny_circuit(n_data: int = 3, layers: int = 2, seed: int = 0, **kw) -> str:
    """A small instance of the same shape, for brute-force checks."""
    kw.setdefault("t_per_layer", 2)
    kw.setdefault("enc_rounds", 2)
    return cultivation_circuit(n_data, layers, seed=seed, **kw)
