"""Pins of the oracle's offline screening and per-shot pre-screen (Sec. 4.2), CPU only."""
import numpy as np
import pytest

from oracle import gates, prescreen, sampler, statevector as sv
from oracle.circuit import parse
from synth import random_circuit, tiny_circuit, workload_circuit


def _noiseless_readout_probs(c):
    rec = []
    sv.run_shot(c, reference=True, record=rec)
    return dict(rec)


@pytest.mark.parametrize("name", ["tiny", "d3_17q_12l"])
def test_decided_measurements_are_deterministic(name):
    """Every measurement that stabiliser tracking decides has p1 in {0, 1} in the noiseless run."""
    c = parse(tiny_circuit(4, 3, seed=2) if name == "tiny" else workload_circuit(name))
    dec = prescreen.decided_measurements(c)
    probs = _noiseless_readout_probs(c)
    assert any(dec.values()) and not all(dec.values())
    for idx, d in dec.items():
        if d:
            assert min(probs[idx], 1 - probs[idx]) < 1e-12


def test_decision_is_basis_independent_on_random_clifford_t():
    """On random Clifford+T circuits, decided => deterministic; and Clifford-only circuits decide
    exactly the measurements the tableau calls deterministic."""
    from oracle import tableau
    for seed in range(4):
        text = random_circuit(6, 100, seed=seed, clifford_only=True, p_meas=0.08, noise=False)
        c = parse(text)
        dec = prescreen.decided_measurements(c)
        tab = tableau.Tableau(c.n)
        for idx, (name, qs) in enumerate(c.ops):
            if name in ("M", "R"):
                det, _ = tab.peek_z(qs[0])
                if name == "M":
                    assert dec[idx] == det
                tab.measure_z(qs[0], forced=0)
            elif name in gates.ONE_Q or name in gates.TWO_Q:
                tab.apply(name, qs)


def _single_fault_cases(c):
    for cid, (kind, qs, idx) in enumerate(c.channels):
        codes = [1] if kind == "XERR" else (range(1, 16) if kind == "DEP2" else range(1, 4))
        for code in codes:
            yield cid, code


def test_single_faults_frame_equals_statevector():
    """For every single fault of a small circuit: the first decided measurement the frame flips has
    p1 = 1 in the faulty state vector, and decided measurements before it have p1 = 0."""
    c = parse(tiny_circuit(3, 2, seed=1))
    dec = prescreen.decided_measurements(c)
    sens, dec_ops = prescreen.sensitivity_matrix(c, dec)
    n_checked = 0
    for cid, code in _single_fault_cases(c):
        flips = sens[cid][code]
        first = next((dec_ops[j] for j in range(len(dec_ops)) if flips[j]), None)
        s = sv.StateVector(c.n)
        fmap = {cid: code}
        for idx, (name, qs) in enumerate(c.ops):
            if name in gates.ONE_Q or name in gates.TWO_Q:
                sv.apply_op(s, name, qs)
            elif name in ("DEP1", "DEP2", "XERR"):
                ch = c.channel_of_op[idx]
                if ch in fmap:
                    for q, pm in zip(qs, gates.fault_paulis(name, fmap[ch])):
                        s.apply1(pm, q)
            else:
                q = qs[0]
                p1 = s.prob1(q)
                if name == "M" and dec[idx]:
                    if idx == first:
                        assert abs(p1 - 1) < 1e-12
                        n_checked += 1
                        break
                    assert p1 < 1e-12
                if p1 > 1 - 1e-12:  # an undecided measurement rejects with certainty
                    break
                s.project(q, 0)
    assert n_checked > 20


def test_frame_and_gf2_routes_agree():
    c = parse(workload_circuit("d3_17q_12l"))
    dec = prescreen.decided_measurements(c)
    faults = sampler.draw_faults(c, p=3e-3, seed=7, shots=range(4096))
    k1 = prescreen.frame_prescreen(c, dec, faults)
    k2 = prescreen.gf2_prescreen(c, dec, faults)
    assert k1 == k2
    kept = sum(k1.values())
    assert 0 < kept < len(k1)


def test_no_false_positives():
    """Every shot the pre-screen removes is rejected by the full simulation (Sec. 4.2)."""
    c = parse(workload_circuit("d3_17q_12l", layers=4))
    dec = prescreen.decided_measurements(c)
    faults = sampler.draw_faults(c, p=5e-3, seed=3, shots=range(512))
    kept = prescreen.frame_prescreen(c, dec, faults)
    removed = [s for s, k in kept.items() if not k][:40]
    assert len(removed) >= 10
    for s in removed:
        status, _, _ = sv.run_shot(c, faults[s], seed=3, shot=s)
        assert status == "rejected"


@pytest.mark.parametrize("seed", range(3))
def test_frame_and_gf2_agree_on_random_circuits(seed):
    c = parse(random_circuit(8, 200, seed=seed, p_meas=0.08, p_reset=0.03))
    dec = prescreen.decided_measurements(c)
    faults = sampler.draw_faults(c, p=2e-2, seed=seed, shots=range(1024))
    assert prescreen.frame_prescreen(c, dec, faults) == prescreen.gf2_prescreen(c, dec, faults)


def _broken_h(orig):
    def f(x, z, name, qs):
        if name != "H":
            orig(x, z, name, qs)
    return f


def _cx_reversed(orig):
    def f(x, z, name, qs):
        if name == "CX":
            orig(x, z, name, (qs[1], qs[0]))
        else:
            orig(x, z, name, qs)
    return f


@pytest.mark.parametrize("plant", [_broken_h, _cx_reversed])
def test_planted_frame_mistake_is_caught(plant):
    """A frame that drops H's X<->Z exchange, or propagates CX the wrong way, disagrees with the
    independent GF(2) route."""
    c = parse(random_circuit(8, 200, seed=1, p_meas=0.08, p_reset=0.03))
    dec = prescreen.decided_measurements(c)
    faults = sampler.draw_faults(c, p=2e-2, seed=1, shots=range(1024))
    ref = prescreen.gf2_prescreen(c, dec, faults)
    orig = prescreen._conj_shape
    prescreen._conj_shape = plant(orig)
    try:
        bad = prescreen.frame_prescreen(c, dec, faults)
    finally:
        prescreen._conj_shape = orig
    assert bad != ref
