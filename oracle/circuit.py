"""Circuit text parser for the oracle (test infrastructure only; shares no code with the library).

Format: one instruction per line, '#' starts a comment.
  QUBITS n                        number of qubits on the line (first instruction)
  H S SDG X Y Z T TDG q           single-qubit gates
  CX c t | CZ a b | SWAP a b      two-qubit gates at any line distance
  M q                             Z measurement, post-selected on outcome 0 (Sec. 4: a shot is
                                  kept only if every measurement returns 0; App. A.3)
  R q                             reset to |0>
  DEP1 q | DEP2 a b               uniform depolarising channel of the rate p (Sec. 4, 4^k-1 Paulis)
  XERR q                          X error channel of rate p (App. A.2, placed before M / after R)
  TICK                            layer marker, no operation
"""
from __future__ import annotations

from dataclasses import dataclass, field

GATES1 = {"H", "S", "SDG", "X", "Y", "Z", "T", "TDG"}
GATES2 = {"CX", "CZ", "SWAP"}
CHANNELS = {"DEP1": 1, "DEP2": 2, "XERR": 1}


@dataclass
class Circuit:
    n: int
    ops: list = field(default_factory=list)          # (name, qubits tuple)
    channel_of_op: dict = field(default_factory=dict)  # op index -> channel id
    readout_of_op: dict = field(default_factory=dict)  # op index -> readout id (M and R)
    channels: list = field(default_factory=list)       # channel id -> (kind, qubits, op index)
    readouts: list = field(default_factory=list)       # readout id -> (kind, qubit, op index)

    @property
    def n_channels(self) -> int:
        return len(self.channels)


def parse(text: str) -> Circuit:
    circ = None
    for lineno, raw in enumerate(text.splitlines(), 1):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        name, args = tok[0].upper(), tok[1:]
        if name == "QUBITS":
            if circ is not None:
                raise ValueError(f"line {lineno}: QUBITS given twice")
            circ = Circuit(n=int(args[0]))
            continue
        if circ is None:
            raise ValueError(f"line {lineno}: QUBITS must come first")
        if name == "TICK":
            continue
        qs = tuple(int(a) for a in args)
        if any(q < 0 or q >= circ.n for q in qs):
            raise ValueError(f"line {lineno}: qubit out of range")
        if name in GATES1 or name in ("M", "R"):
            want = 1
        elif name in GATES2:
            want = 2
        elif name in CHANNELS:
            want = CHANNELS[name]
        else:
            raise ValueError(f"line {lineno}: unknown instruction {name}")
        if len(qs) != want:
            raise ValueError(f"line {lineno}: {name} takes {want} qubit(s)")
        if want == 2 and qs[0] == qs[1]:
            raise ValueError(f"line {lineno}: {name} on one qubit twice")
        idx = len(circ.ops)
        circ.ops.append((name, qs))
        if name in CHANNELS:
            circ.channel_of_op[idx] = len(circ.channels)
            circ.channels.append((name, qs, idx))
        elif name in ("M", "R"):
            circ.readout_of_op[idx] = len(circ.readouts)
            circ.readouts.append((name, qs[0], idx))
    if circ is None:
        raise ValueError("empty circuit")
    return circ
