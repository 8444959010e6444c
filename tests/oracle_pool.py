"""Runs the CPU oracle (FP64 NumPy MPS) over many shots in a process pool (test infrastructure).

The pool is started with the "spawn" method: a process forked after the parent has touched the GPU
can hang, and spawned children import nothing of the CUDA path.  Each child parses the circuit and
builds the noiseless reference state once; a task is one shot with its fault list.
"""
from __future__ import annotations

import multiprocessing as mp
import os

_STATE = {}


def _init(text, chi_max, cutoff, seed):
    from oracle import mps as omps
    from oracle.circuit import parse
    circ = parse(text)
    _, ref, _ = omps.run_shot(circ, reference=True, chi_max=chi_max, cutoff=cutoff)
    _STATE.update(circ=circ, ref=ref, chi_max=chi_max, cutoff=cutoff, seed=seed)


def _shot(task):
    from oracle import mps as omps
    shot, faults = task
    rec = []
    st, psi, abort = omps.run_shot(_STATE["circ"], faults, seed=_STATE["seed"], shot=shot,
                                   chi_max=_STATE["chi_max"], cutoff=_STATE["cutoff"], record=rec)
    f = omps.fidelity(_STATE["ref"], psi) if st == "accepted" else None
    return shot, st, abort, f, len(faults), [p1 for _, p1 in rec], psi.discarded


def oracle_shots(text, shots, faults, *, seed, chi_max=1 << 30, cutoff=0.0, procs=None):
    """{shot: (status, abort_op, fidelity, weight, readout p1 list, discarded)} from the oracle MPS."""
    shots = [int(s) for s in shots]
    if not shots:
        return {}
    procs = procs or max(1, min(len(shots), os.cpu_count() or 1, 32))
    old = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"  # one BLAS thread per child, inherited at spawn
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs, initializer=_init, initargs=(text, chi_max, cutoff, seed)) as pool:
            out = pool.map(_shot, [(s, list(faults[s])) for s in shots], chunksize=1)
    finally:
        if old is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = old
    return {s: rest for s, *rest in out}
