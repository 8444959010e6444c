"""Fault sampling and the Pauli pre-screen on the GPU against the oracle: bit-exact."""
import numpy as np
import pytest
import torch

from oracle import prescreen, sampler
from oracle.circuit import parse
from synth import random_circuit, workload_circuit

from gpu_common import dev_shots, kept_bits, lib_ready

pytestmark = pytest.mark.gpu


def _oracle_faults(text, p, seed, shots, weight=-1):
    return sampler.draw_faults(parse(text), p=p, seed=seed, shots=shots, fault_weight=weight)


@pytest.mark.parametrize("p", [1e-3, 2e-2])
def test_fault_lists_bit_exact(p):
    q = lib_ready()
    text = workload_circuit("d3_17q_12l")
    c = q.Circuit(text)
    rng = np.random.default_rng(5)
    shots = np.concatenate([np.arange(0, 700), rng.integers(0, 10**10, size=300)])
    count, chan, code = q.qc_sample_faults(c, dev_shots(shots), p=p, seed=1234, max_faults=64)
    count, chan, code = count.cpu().numpy(), chan.cpu().numpy(), code.cpu().numpy()
    ref = _oracle_faults(text, p, 1234, shots)
    for i, s in enumerate(shots):
        exp = ref[int(s)]
        assert count[i] == len(exp)
        got = list(zip(chan[i, :count[i]].tolist(), code[i, :count[i]].tolist()))
        assert got == exp, (s, got, exp)


@pytest.mark.parametrize("w", [0, 1, 3, 7])
def test_exact_weight_fault_lists(w):
    q = lib_ready()
    text = workload_circuit("d3_17q_12l", layers=4)
    c = q.Circuit(text)
    shots = np.arange(0, 257) * 7919
    count, chan, code = q.qc_sample_faults(c, dev_shots(shots), p=0.0, seed=77, fault_weight=w, max_faults=16)
    count, chan, code = count.cpu().numpy(), chan.cpu().numpy(), code.cpu().numpy()
    ref = _oracle_faults(text, 0.0, 77, shots, weight=w)
    for i, s in enumerate(shots):
        assert count[i] == w
        assert list(zip(chan[i, :w].tolist(), code[i, :w].tolist())) == ref[int(s)]


def _check_prescreen(text, p, seed, shot0, nshots, w_max=15):
    q = lib_ready()
    c = q.Circuit(text)
    out = q.pauli_prescreen(c, shot0, nshots, p=p, seed=seed, w_max=w_max)
    got = kept_bits(out["kept_mask"], nshots)
    oc = parse(text)
    shots = range(shot0, shot0 + nshots)
    faults = sampler.draw_faults(oc, p=p, seed=seed, shots=shots)
    kept = prescreen.frame_prescreen(oc, prescreen.decided_measurements(oc), faults)
    exp = np.array([kept[s] for s in shots], dtype=bool)
    assert np.array_equal(got, exp)
    surv = out["survivors"].cpu().numpy()
    assert out["n_kept"] == exp.sum()
    assert np.array_equal(surv, np.array([s for s in shots if kept[s]], dtype=np.int64))
    hd = np.zeros(w_max + 1, dtype=np.uint64)
    hk = np.zeros(w_max + 1, dtype=np.uint64)
    for s in shots:
        w = min(len(faults[s]), w_max)
        hd[w] += 1
        hk[w] += kept[s]
    assert np.array_equal(out["hist_drawn"], hd)
    assert np.array_equal(out["hist_kept"], hk)
    return exp


def test_prescreen_workload_ragged_tail():
    exp = _check_prescreen(workload_circuit("d3_17q_12l"), 3e-3, 9, 0, 20000 + 37)
    assert 0 < exp.sum() < len(exp)


def test_prescreen_offset_and_small():
    _check_prescreen(workload_circuit("d3_17q_12l"), 1e-2, 3, 64 * 1000, 1000)
    _check_prescreen(workload_circuit("d3_17q_12l"), 1e-2, 3, 64 * 5, 1)


def test_prescreen_zero_rate_keeps_everything():
    exp = _check_prescreen(workload_circuit("d3_17q_12l"), 0.0, 1, 0, 640)
    assert exp.all()


@pytest.mark.parametrize("seed", [0, 1])
def test_prescreen_random_circuit(seed):
    _check_prescreen(random_circuit(9, 400, seed=seed, p_meas=0.08, p_reset=0.04), 2e-2, seed, 0, 4096 + 5)


def test_prescreen_empty_and_invalid():
    q = lib_ready()
    c = q.Circuit(workload_circuit("d3_17q_12l", layers=2))
    out = q.pauli_prescreen(c, 0, 0, p=1e-3, seed=1)
    assert out["n_kept"] == 0
    with pytest.raises(q.QcError):
        q.pauli_prescreen(c, 3, 64, p=1e-3, seed=1)
    with pytest.raises(q.QcError):
        q.pauli_prescreen(c, 0, 64, p=1.5, seed=1)


@pytest.mark.parametrize("p", [1e-3, 2e-4])
def test_prescreen_full_size_sampled(p):
    """The 49-qubit, 200-layer pre-screen workload at 1e8 shots, in the launch the benchmark
    uses; 384 sampled shots are recomputed by the oracle (at p = 1e-3 nearly all are discarded,
    p = 2e-4 keeps about 1 % so kept shots are sampled too)."""
    q = lib_ready()
    text = workload_circuit("d5_49q_200l")
    c = q.Circuit(text)
    n = 10**8
    out = q.pauli_prescreen(c, 0, n, p=p, seed=0, survivors_capacity=0)
    mask = out["kept_mask"].cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.integers(0, n, size=384).tolist()) | {0, n - 1})
    oc = parse(text)
    faults = sampler.draw_faults(oc, p=p, seed=0, shots=sample)
    kept = prescreen.frame_prescreen(oc, prescreen.decided_measurements(oc), faults)
    for s in sample:
        assert bool((int(mask[s >> 6]) >> (s & 63)) & 1) == kept[s], s
    assert out["hist_drawn"].sum() == n
    assert out["hist_kept"].sum() == sum(int(w).bit_count() for w in mask)


@pytest.mark.parametrize("w", [1, 3, 5])
def test_prescreen_fixed_weight_bit_exact(w):
    """Subset sampling (Sec. 4.1): every shot has exactly w faults; kept flags equal the oracle's."""
    q = lib_ready()
    text = workload_circuit("d5_49q_60l", layers=10)
    c = q.Circuit(text)
    n = 64 * 40 + 17
    out = q.pauli_prescreen(c, 64 * 3, n, p=0.0, seed=21, fault_weight=w)
    got = kept_bits(out["kept_mask"], n)
    oc = parse(text)
    shots = range(64 * 3, 64 * 3 + n)
    faults = sampler.draw_faults(oc, p=0.0, seed=21, shots=shots, fault_weight=w)
    kept = prescreen.frame_prescreen(oc, prescreen.decided_measurements(oc), faults)
    exp = np.array([kept[s] for s in shots], dtype=bool)
    assert np.array_equal(got, exp)
    assert out["n_kept"] == exp.sum()
    assert np.array_equal(out["survivors"].cpu().numpy(), np.array([s for s in shots if kept[s]], dtype=np.int64))
    assert out["hist_drawn"][w] == n and out["hist_kept"][w] == exp.sum()
