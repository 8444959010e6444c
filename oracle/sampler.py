"""The per-shot sampling pipeline, test infrastructure only (Sec. 4).

For each shot: draw its fault configuration, apply the offline pre-screen (Sec. 4.2), and if it
survives simulate it with early stop at the first measurement returning 1 (Sec. 4.3).  Every shot
ends discarded, accepted and correct, or accepted and logically wrong (Sec. 4); counts are kept
per fault weight w (Eq. estimators): n_w (all drawn shots, pre-screened ones included), n_w^acc
and n_w^err.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import mps as mps_mod
from . import statevector as sv_mod
from .philox import sample_faults_bernoulli, sample_faults_exact
from .prescreen import decided_measurements, frame_prescreen


@dataclass
class ShotResult:
    shot: int
    weight: int
    kept: bool            # survived the pre-screen
    accepted: bool
    logical_error: bool
    fidelity: float
    abort_op: int | None
    discarded: float = 0.0


def channel_kinds(circ):
    return [kind for kind, _, _ in circ.channels]


def draw_faults(circ, *, p, seed, shots, fault_weight=-1):
    kinds = channel_kinds(circ)
    if fault_weight < 0:
        return sample_faults_bernoulli(seed, kinds, p, shots)
    return {int(s): sample_faults_exact(seed, kinds, fault_weight, int(s)) for s in shots}


def sample(circ, *, p, seed, shots, engine="sv", chi_max=1 << 30, cutoff=0.0, tau=1e-8,
           fault_weight=-1, prescreen=True):
    shots = [int(s) for s in shots]
    faults = draw_faults(circ, p=p, seed=seed, shots=shots, fault_weight=fault_weight)
    decided = decided_measurements(circ)
    kept = frame_prescreen(circ, decided, faults) if prescreen else {s: True for s in shots}
    if engine == "sv":
        _, ref, _ = sv_mod.run_shot(circ, reference=True)
    else:
        _, ref, _ = mps_mod.run_shot(circ, reference=True, chi_max=chi_max, cutoff=cutoff)
    counts = {}
    results = []
    for s in shots:
        w = len(faults[s])
        c = counts.setdefault(w, [0, 0, 0])
        c[0] += 1
        if not kept[s]:
            results.append(ShotResult(s, w, False, False, False, float("nan"), None))
            continue
        if engine == "sv":
            status, st, abort = sv_mod.run_shot(circ, faults[s], seed=seed, shot=s)
            disc = 0.0
        else:
            status, st, abort = mps_mod.run_shot(circ, faults[s], seed=seed, shot=s,
                                                 chi_max=chi_max, cutoff=cutoff)
            disc = st.discarded
        if status != "accepted":
            results.append(ShotResult(s, w, True, False, False, float("nan"), abort, disc))
            continue
        f = sv_mod.fidelity(ref, st) if engine == "sv" else mps_mod.fidelity(ref, st)
        err = (1.0 - f) > tau
        c[1] += 1
        c[2] += int(err)
        results.append(ShotResult(s, w, True, True, err, f, None, disc))
    return {w: tuple(v) for w, v in sorted(counts.items())}, results
