"""Pins of the oracle simulators against closed forms, the CHP tableau and each other (CPU)."""
import math

import numpy as np
import pytest

from oracle import gates, mps, statevector as sv, tableau
from oracle.circuit import parse
from synth import random_circuit, workload_circuit


def _sv(n, ops):
    s = sv.StateVector(n)
    for name, qs in ops:
        sv.apply_op(s, name, qs)
    return s


def test_closed_form_ancilla_marginal():
    """H T H |0>: P(0) = cos^2(pi/8)."""
    s = _sv(1, [("H", (0,)), ("T", (0,)), ("H", (0,))])
    assert abs((1 - s.prob1(0)) - math.cos(math.pi / 8) ** 2) < 1e-15
    m = mps.MPS(1)
    for g in ("H", "T", "H"):
        m.apply1(gates.ONE_Q[g], 0)
    assert abs((1 - m.prob1(0)) - math.cos(math.pi / 8) ** 2) < 1e-15


@pytest.mark.parametrize("pauli,expect", [("X", 0.5), ("Y", 0.5), ("Z", 0.0)])
def test_closed_form_t_state_overlaps(pauli, expect):
    """|<T|P|T>|^2 for |T> = T|+> (Sec. 1; App. A.3: Pauli faults move the overlap far from 1)."""
    t = _sv(1, [("H", (0,)), ("T", (0,))])
    tp = _sv(1, [("H", (0,)), ("T", (0,)), (pauli, (0,))])
    assert abs(sv.fidelity(t, tp) - expect) < 1e-15


def _tableau_vs_statevector(text):
    c = parse(text)
    tab = tableau.Tableau(c.n)
    s = sv.StateVector(c.n)
    checked = 0
    for name, qs in c.ops:
        if name in gates.ONE_Q or name in gates.TWO_Q:
            tab.apply(name, qs)
            sv.apply_op(s, name, qs)
        elif name in ("M", "R"):
            q = qs[0]
            det, val = tab.peek_z(q)
            p1 = s.prob1(q)
            if det:
                assert abs(p1 - val) < 1e-12
                out = val
            else:
                assert abs(p1 - 0.5) < 1e-12
                out = 0
            tab.measure_z(q, forced=out)
            s.project(q, out)
            if name == "R" and out == 1:
                tab.apply("X", (q,))
                s.apply1(gates.X, q)
            checked += 1
    return checked


@pytest.mark.parametrize("seed", range(6))
def test_statevector_matches_tableau_on_clifford(seed):
    text = random_circuit(7, 120, seed=seed, clifford_only=True, p_meas=0.1, p_reset=0.05, noise=False)
    assert _tableau_vs_statevector(text) > 5


@pytest.mark.parametrize("seed", range(6))
def test_mps_exact_matches_statevector(seed):
    """Untruncated MPS = state vector (Sec. 3.1: exact regime), incl. SWAP routing at distance <= 3."""
    c = parse(random_circuit(8, 150, seed=seed, max_dist=3, noise=False))
    s = sv.StateVector(c.n)
    m = mps.MPS(c.n, cutoff=0.0)
    for name, qs in c.ops:
        if name in gates.ONE_Q:
            s.apply1(gates.ONE_Q[name], qs[0]); m.apply1(gates.ONE_Q[name], qs[0])
        elif name in gates.TWO_Q:
            s.apply2(gates.TWO_Q[name], *qs); m.apply2(gates.TWO_Q[name], *qs)
    assert np.allclose(s.vector(), m.vector(), atol=1e-12)
    for k, chi in enumerate(m.bond_dims()):
        assert chi <= 2 ** min(k + 1, c.n - k - 1)  # Sec. 3.1: chi_k <= 2^min(k, N-k)


def test_mps_readouts_match_statevector_on_workload():
    c = parse(workload_circuit("d3_17q_12l"))
    r1, r2 = [], []
    sv.run_shot(c, reference=True, record=r1)
    mps.run_shot(c, reference=True, record=r2, cutoff=1e-12)
    assert len(r1) == len(r2) == len(c.readouts)
    assert max(abs(a[1] - b[1]) for a, b in zip(r1, r2)) < 1e-10


def test_mps_truncation_rule_and_discarded_weight():
    c = parse(random_circuit(10, 300, seed=3, max_dist=2, noise=False, one_q=("H", "T", "S")))
    _, exact, _ = mps.run_shot(c, reference=True)
    _, trunc, _ = mps.run_shot(c, reference=True, chi_max=4, cutoff=0.0)
    assert max(trunc.bond_dims()) <= 4
    f = mps.fidelity(exact, trunc)
    assert trunc.discarded > 0
    assert 1 - f <= 2 * trunc.discarded + 1e-12
    assert abs(trunc.norm2() - 1) < 1e-12
    # with chi_max at least the Schmidt rank nothing is discarded
    _, big, _ = mps.run_shot(c, reference=True, chi_max=64, cutoff=1e-14)
    assert big.discarded < 1e-20 and abs(mps.fidelity(exact, big) - 1) < 1e-12


def test_truncation_rule_counts():
    m = mps.MPS(2, chi_max=3, cutoff=0.05)
    s = np.array([0.8, 0.5, 0.3, 0.1])  # squares .64 .25 .09 .01, total .99
    r = m._truncate(s)
    # tail after 2 = .10/.99 > .05; after 3 = .01/.99 <= .05 -> r = 3
    assert r == 3 and abs(m.discarded - 0.01 / 0.99) < 1e-15
    m2 = mps.MPS(2, chi_max=2, cutoff=0.05)
    assert m2._truncate(s) == 2
    m3 = mps.MPS(2, chi_max=8, cutoff=0.0)
    assert m3._truncate(np.array([1.0, 0.0])) == 1


def test_overlap_sweep_matches_dense():
    c = parse(random_circuit(6, 80, seed=4, noise=False))
    _, a, _ = mps.run_shot(c, reference=True)
    c2 = parse(random_circuit(6, 80, seed=5, noise=False))
    _, b, _ = mps.run_shot(c2, reference=True)
    assert abs(mps.overlap(a, b) - np.vdot(a.vector(), b.vector())) < 1e-12


def test_truncation_rule_and_degenerate_flag_on_crafted_spectra():
    """The written truncation rule on spectra whose outcome follows from its definition: the kept count
    is the smallest r with tail sum s_i^2 (i >= r) <= cutoff x total, capped by chi_max; the cut is
    flagged degenerate exactly when the last kept and the first dropped value agree to 1e-8 relative."""
    from oracle.mps import MPS
    flat = np.full(8, 1 / np.sqrt(8))
    m = MPS(2, chi_max=4, cutoff=0.0)
    assert m._truncate(flat) == 4 and m.degenerate_cuts == 1          # cut inside a flat spectrum
    assert abs(m.discarded - 0.5) < 1e-15
    m = MPS(2, chi_max=4, cutoff=0.0)
    gap = np.array([0.6, 0.5, 0.4, 0.3, 0.2, 0.1])
    assert m._truncate(gap) == 4 and m.degenerate_cuts == 0           # clear gap at the cut
    m = MPS(2, chi_max=4, cutoff=0.0)
    near = np.array([0.5, 0.5, 0.5, 0.5 * (1 + 5e-9), 0.5, 0.1])
    near = -np.sort(-near)
    assert m._truncate(near) == 4 and m.degenerate_cuts == 1          # within 1e-8 relative
    m = MPS(2, chi_max=4, cutoff=0.0)
    apart = np.array([0.5 * (1 + 3e-8), 0.5 * (1 + 2e-8), 0.5 * (1 + 1e-8 + 1e-9), 0.5 * (1 + 1e-8 + 1e-9), 0.5, 0.1])
    assert m._truncate(apart) == 4 and m.degenerate_cuts == 0         # 1.1e-8 apart: not flagged
    m = MPS(2, chi_max=8, cutoff=0.1)
    s = np.sqrt(np.array([0.5, 0.3, 0.12, 0.05, 0.03]))
    assert m._truncate(s) == 3 and abs(m.discarded - 0.08) < 1e-12    # tail 0.08 <= 0.1, tail at 2 is 0.2
    m = MPS(2, chi_max=8, cutoff=0.0)
    z = np.array([1.0, 0.0, 0.0])
    assert m._truncate(z) == 1 and m.degenerate_cuts == 0             # exact zeros: tail 0 <= 0 at r = 1
