"""Oracle parity of the benchmark's own engine path and of intermediate quantities (Sec. 3.1, 4, 4.3).

* The one-warp-per-shot engine on the 49-qubit workload in the launch the benchmark times (more
  shots than SMs, complex64, chi_max 256, cutoff 1e-10): there every 64-wide theta is rotated in
  global memory by the blocked Jacobi.  Fidelity and every readout probability at 1e-4 absolute
  (the complex64 tolerance), on shots sampled across the batch.
* The blocked Jacobi forced at complex128 (a small shared-memory work area) on a 6-layer circuit
  of the 49-qubit workload's shape: fidelity and readout probabilities at 1e-10.
* The large-bond workloads (check layers up to bond 128 and 256) on their true 2-layer prefixes.
* Per-readout Born probabilities of the default (one CTA per shot) complex128 engine at 1e-10.
* Logical-error and acceptance rates of the 17-qubit, 1,000-shot configuration against the
  oracle's own pre-screen + MPS pipeline, within binomial intervals.
* The Jacobi sweep limit: a cap of one sweep makes splits run out, which ends those shots with
  per-shot status QC_ENOCONV while the call itself succeeds.
"""
import math

import numpy as np
import pytest
import torch

from oracle import prescreen, sampler
from oracle.circuit import parse
from synth import workload_circuit

from gpu_common import dev_shots, lib_ready
from oracle_pool import oracle_shots

pytestmark = pytest.mark.gpu

QC_ENOCONV = -4


def _n_readouts(c):
    inf = c.info()
    return int(inf["n_measurements"] + inf["n_resets"])


def _compare(res, rec, ref, ftol, ptol, allow_flip=0):
    """Per shot: status, abort position, fidelity and every readout probability against the oracle.
    Returns the number of status flips (a c64 draw within ptol of p1 may decide differently)."""
    flips = 0
    for i, r in enumerate(res):
        st, abort, f, w, p1, _ = ref[int(r["shot"])]
        assert r["weight"] == w
        assert r["status"] in (0, 1), r
        got = rec[i][~np.isnan(rec[i])]
        if (r["status"] == 0) != (st == "accepted"):
            flips += 1
            continue
        assert len(got) == min(len(p1), rec.shape[1]), (int(r["shot"]), len(got), len(p1))
        np.testing.assert_allclose(got, np.asarray(p1[: len(got)]), rtol=0, atol=ptol)
        if st == "accepted":
            assert abs(r["fidelity"] - f) < ftol, (r, f)
        else:
            assert r["abort_op"] == abort
    assert flips <= allow_flip, flips
    return flips


def test_benchmark_launch_warp_engine_blocked_jacobi_c64():
    """The benchmark's kernel and launch (one warp per shot, 24 KB work area, capacity bucket 64) on a
    10-layer circuit of the 49-qubit workload's shape (its own seeded draw, which reaches 64-wide
    theta early); 24 shots sampled across a 200-shot batch."""
    q = lib_ready()
    text = workload_circuit("d5_49q_60l", layers=10)
    c = q.Circuit(text)
    p, seed = 1e-3, 0
    shots = q.pauli_prescreen(c, 0, 64 * 4096, p=p, seed=seed)["survivors"][:200]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert shots.numel() > nsm  # more shots than SMs: the engine picks one warp per shot
    K = _n_readouts(c)
    _, res, rec = q.mps_sample_batch_traced(c, shots, p=p, seed=seed, chi_max=256, cutoff=1e-10,
                                            precision=q.QC_C64, readout_k=K)
    idx = np.linspace(0, len(res) - 1, 24).astype(int)
    pick = [int(res["shot"][i]) for i in idx]
    faults = sampler.draw_faults(parse(text), p=p, seed=seed, shots=pick)
    ref = oracle_shots(text, pick, faults, seed=seed, chi_max=256, cutoff=1e-10)
    _compare(res[idx], rec[idx], ref, 1e-4, 1e-4, allow_flip=1)
    # the compared shots went through the global-memory blocked Jacobi (64-wide theta)
    assert (res["gmem_updates"][idx] > 0).mean() >= 0.5, res["gmem_updates"][idx]
    assert (res["chi_peak"] >= 32).any()


def test_blocked_jacobi_forced_c128(monkeypatch):
    """A 12 KB work area per warp at complex128 on a 6-layer circuit of the 49-qubit workload's shape: every
    64-wide theta goes to global memory and is rotated by the blocked Jacobi in blocks of 3 columns
    (12 KB holds ~430 complex128 elements next to the fixed arrays, 2 blocks x 65 rows each fit)."""
    monkeypatch.setenv("QCMPS_ENGINE", "warp")
    monkeypatch.setenv("QCMPS_SMEM_KB", "12")
    q = lib_ready()
    text = workload_circuit("d5_49q_60l", layers=6)
    c = q.Circuit(text)
    p, seed = 2e-3, 13
    shots = q.pauli_prescreen(c, 0, 64 * 64, p=p, seed=seed)["survivors"][:16]
    K = _n_readouts(c)
    _, res, rec = q.mps_sample_batch_traced(c, shots, p=p, seed=seed, chi_max=256, cutoff=1e-12,
                                            precision=q.QC_C128, readout_k=K)
    pick = [int(s) for s in res["shot"]]
    faults = sampler.draw_faults(parse(text), p=p, seed=seed, shots=pick)
    ref = oracle_shots(text, pick, faults, seed=seed, chi_max=256, cutoff=1e-12)
    _compare(res, rec, ref, 1e-10, 1e-10)
    assert (res["gmem_updates"] > 0).all(), res["gmem_updates"]


@pytest.mark.parametrize("prec,tol", [(1, 1e-10), (0, 1e-4)])
def test_readout_probabilities_default_launch(prec, tol):
    """Few shots (one CTA per shot, the whole split in shared memory): every readout's p1."""
    q = lib_ready()
    text = workload_circuit("d3_17q_12l")
    c = q.Circuit(text)
    p, seed = 3e-3, 21
    shots = q.pauli_prescreen(c, 64 * 100, 64 * 6, p=p, seed=seed)["survivors"][:24]
    K = _n_readouts(c)
    _, res, rec = q.mps_sample_batch_traced(c, shots, p=p, seed=seed, chi_max=32, cutoff=1e-12, precision=prec,
                                            readout_k=K)
    pick = [int(s) for s in res["shot"]]
    faults = sampler.draw_faults(parse(text), p=p, seed=seed, shots=pick)
    ref = oracle_shots(text, pick, faults, seed=seed, chi_max=32, cutoff=1e-12)
    _compare(res, rec, ref, 1e-10 if prec == 1 else 1e-4, tol, allow_flip=0 if prec == 1 else 1)
    # a record shorter than the circuit's readouts is a prefix of the same record
    _, _, rec4 = q.mps_sample_batch_traced(c, shots, p=p, seed=seed, chi_max=32, cutoff=1e-12, precision=prec,
                                           readout_k=4)
    np.testing.assert_array_equal(rec4, rec[:, :4])


def _binomial_halfwidth(k, n, z=3.3):
    """Normal-approximation half width of a binomial rate (z = 3.3: two-sided 0.1 %), with the
    1/n floor of a rate estimated from n trials."""
    r = k / n if n else 0.0
    return z * math.sqrt(max(r * (1 - r), 1.0 / n) / n) + 1.0 / n if n else 1.0


def test_c1_rates_within_binomial_intervals():
    """17 qubits, 12 layers, p = 1e-3, chi_max 32, cutoff 1e-12, complex128, 1,000 drawn shots:
    acceptance and logical-error rates per fault weight, GPU (pre-screen + engine) against the oracle
    (frame pre-screen + FP64 MPS), agree within binomial intervals; with the same random numbers the
    per-shot decisions are in fact identical."""
    q = lib_ready()
    text = workload_circuit("d3_17q_12l")
    c = q.Circuit(text)
    p, seed, n = 1e-3, 0, 1000
    pre = q.pauli_prescreen(c, 0, n, p=p, seed=seed, w_max=15)
    counts, res = q.mps_sample_batch(c, pre["survivors"], p=p, seed=seed, chi_max=32, cutoff=1e-12,
                                     precision=q.QC_C128, w_max=15)
    counts[:, 0] = pre["hist_drawn"]
    oc = parse(text)
    faults = sampler.draw_faults(oc, p=p, seed=seed, shots=range(n))
    kept = prescreen.frame_prescreen(oc, prescreen.decided_measurements(oc), faults)
    surv = [s for s in range(n) if kept[s]]
    assert surv == [int(s) for s in pre["survivors"].cpu()]
    ref = oracle_shots(text, surv, faults, seed=seed, chi_max=32, cutoff=1e-12)
    oc_counts = np.zeros_like(counts)
    for s in range(n):
        w = min(len(faults[s]), 15)
        oc_counts[w, 0] += 1
        if s in ref and ref[s][0] == "accepted":
            oc_counts[w, 1] += 1
            oc_counts[w, 2] += int(1.0 - ref[s][2] > 1e-8)
    assert np.array_equal(counts[:, 0], oc_counts[:, 0])
    for w in range(16):
        nw = int(counts[w, 0])
        if nw == 0:
            continue
        for col in (1, 2):  # acceptance rate, logical-error rate (per drawn shot)
            hw = _binomial_halfwidth(int(oc_counts[w, col]), nw)
            assert abs(int(counts[w, col]) - int(oc_counts[w, col])) / nw <= hw, (w, col, counts[w], oc_counts[w])
    same = sum(1 for r in res if (r["status"] == 0) == (ref[int(r["shot"])][0] == "accepted") and
               (r["status"] != 0 or bool(r["logical_error"]) == (1.0 - ref[int(r["shot"])][2] > 1e-8)))
    assert same >= len(res) - 1, (same, len(res))
    assert counts[:, 1].sum() > 0.5 * n


def test_sweep_cap_ends_shots_with_enoconv():
    """A Jacobi limit of one sweep cannot orthogonalise an entangled theta: the shot ends with
    QC_ENOCONV in its record, is counted as drawn but not accepted, and the call returns QC_OK."""
    q = lib_ready()
    text = workload_circuit("d3_17q_12l", layers=3)
    c = q.Circuit(text)
    shots = dev_shots(list(range(0, 40)))
    # warm the cached reference state with the default limit first
    q.mps_sample_batch(c, shots[:1], p=0.0, seed=3, chi_max=32, cutoff=1e-12, precision=q.QC_C64)
    counts, res, _ = q.mps_sample_batch_traced(c, shots, p=0.0, seed=3, chi_max=32, cutoff=1e-12,
                                               precision=q.QC_C64, sweep_cap=1)
    assert (res["status"] == QC_ENOCONV).all(), np.unique(res["status"])
    assert counts[:, 0].sum() == 40 and counts[:, 1].sum() == 0
    # the same shots with the default limit converge
    counts2, res2 = q.mps_sample_batch(c, shots, p=0.0, seed=3, chi_max=32, cutoff=1e-12, precision=q.QC_C64)
    assert (res2["status"] == 0).all()


@pytest.mark.parametrize("name,prec,tol", [("d5_49q_60l_b128", 0, 1e-4), ("d5_49q_60l_b128", 1, 1e-10),
                                           ("d5_49q_60l_b256", 0, 1e-4)])
def test_large_bond_workloads_match_oracle(name, prec, tol):
    """The large-bond workloads (encoded bond 64, check layers up to bond 128 / 256) on their true
    2-layer prefix: one CTA per shot with the theta of the widest splits in global memory; fidelity and
    every readout probability against the oracle."""
    q = lib_ready()
    text = workload_circuit(name, prefix_layers=2)
    c = q.Circuit(text)
    p, seed = 2e-3, 5
    shots = q.pauli_prescreen(c, 0, 64 * 64, p=p, seed=seed)["survivors"][:10]
    K = _n_readouts(c)
    _, res, rec = q.mps_sample_batch_traced(c, shots, p=p, seed=seed, chi_max=256, cutoff=1e-10, precision=prec,
                                            readout_k=K)
    pick = [int(s) for s in res["shot"]]
    faults = sampler.draw_faults(parse(text), p=p, seed=seed, shots=pick)
    ref = oracle_shots(text, pick, faults, seed=seed, chi_max=256, cutoff=1e-10)
    _compare(res, rec, ref, tol, tol, allow_flip=0 if prec == 1 else 1)
    assert res["chi_peak"].max() >= 64, res["chi_peak"]
    assert (res["status"] >= 0).all()
