"""Pins of the oracle's random-number contract (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox_kat.txt")):
        line = line.split("#", 1)[0].split()
        if line:
            v = [int(t, 16) for t in line]
            rows.append((v[:6], v[6:]))
    return rows


@pytest.mark.parametrize("inp,out", _kat())
def test_philox_known_answers(inp, out):
    x = philox.philox4x32_10(*inp)
    assert [int(v) for v in x] == out


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2**32, size=(4, 50), dtype=np.uint64)
    k = rng.integers(0, 2**32, size=2, dtype=np.uint64)
    xs = philox.philox4x32_10(c[0], c[1], c[2], c[3], k[0], k[1])
    for j in range(50):
        xj = philox.philox4x32_10(c[0, j], c[1, j], c[2, j], c[3, j], k[0], k[1])
        assert [int(v[j]) for v in xs] == [int(v) for v in xj]


def test_thresholds_closed_form():
    for p in (1e-4, 1e-3, 5e-3, 0.1):
        t1, tg = philox.thresholds(p)
        assert t1 == math.floor(p * 2**32)
        q = t1 / 2**32
        for s in (0, 1, 7, 63):
            exact = (1 - (1 - q) ** (s + 1)) * 2**32
            assert abs(int(tg[s]) - exact) <= 2.0
        assert np.all(np.diff(tg.astype(np.int64)) >= 0)
        assert int(tg[0]) == t1 or abs(int(tg[0]) - t1) <= 1


def test_thresholds_zero_rate():
    t1, tg = philox.thresholds(0.0)
    assert t1 == 0 and not tg.any()
    out = philox.sample_faults_bernoulli(3, ["DEP1"] * 100, 0.0, range(200))
    assert all(len(v) == 0 for v in out.values())


def test_lane_rate_and_independence():
    """Faulted lanes are independent Bernoulli(p): rate within 5 sigma, no lane bias, pair
    co-occurrence at p^2 (geometric gaps reproduce iid lanes)."""
    p = 0.02
    kinds = ["DEP1"] * 256
    shots = range(64 * 64)
    faults = philox.sample_faults_bernoulli(11, kinds, p, shots)
    mat = np.zeros((len(shots), len(kinds)), dtype=np.uint8)
    for s, fl in faults.items():
        for c, _ in fl:
            mat[s, c] = 1
    n = mat.size
    rate = mat.mean()
    assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / n)
    lane_rate = mat.reshape(64, 64, -1).mean(axis=(0, 2))  # per lane
    assert lane_rate.max() < p + 6 * math.sqrt(p / (64 * 256))
    pair = (mat[0::2] & mat[1::2]).mean()
    assert abs(pair - p * p) < 6 * math.sqrt(p * p / (n / 2))


def test_pauli_codes_uniform():
    kinds = ["DEP2"] * 64 + ["DEP1"] * 64 + ["XERR"] * 8
    faults = philox.sample_faults_bernoulli(5, kinds, 0.05, range(64 * 64))
    c2 = np.zeros(16)
    c1 = np.zeros(4)
    for fl in faults.values():
        for c, code in fl:
            if kinds[c] == "DEP2":
                c2[code] += 1
            elif kinds[c] == "DEP1":
                c1[code] += 1
            else:
                assert code == 1
    assert c2[0] == 0 and c1[0] == 0
    e2 = c2[1:].sum() / 15
    assert np.all(np.abs(c2[1:] - e2) < 6 * math.sqrt(e2))
    e1 = c1[1:].sum() / 3
    assert np.all(np.abs(c1[1:] - e1) < 6 * math.sqrt(e1))


def test_exact_weight_sampling():
    kinds = ["DEP1"] * 40
    counts = np.zeros(40)
    for s in range(3000):
        fl = philox.sample_faults_exact(9, kinds, 3, s)
        chans = [c for c, _ in fl]
        assert len(chans) == 3 and len(set(chans)) == 3 and chans == sorted(chans)
        for c in chans:
            counts[c] += 1
    e = 3000 * 3 / 40
    assert np.all(np.abs(counts - e) < 6 * math.sqrt(e))
    assert philox.sample_faults_exact(9, kinds, 0, 5) == []
    assert len(philox.sample_faults_exact(9, kinds, 40, 5)) == 40


def test_readout_uniform():
    u = np.array([philox.readout_uniform(2, k, s) for k in range(20) for s in range(500)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))
    # 53-bit resolution: values are multiples of 2^-53
    assert all((x * 2**53) == int(x * 2**53) for x in u[:100])


@pytest.mark.parametrize("p", [1e-3, 0.05, 0.3])
def test_vectorised_fault_sampler_equals_scalar_contract(p):
    """The vectorised Bernoulli sampler (every test's fault source) against the scalar statement of
    the contract: for every channel and every word, the lanes of `faulted_lanes` (first lane from the
    word draw, then geometric skips while the next lane stays below 64) and the Pauli of each lane
    from `pauli_code`.  At p = 0.3 a word holds ~19 faulted lanes, so the skip counter passes several
    Philox blocks (k >> 2 > 0) and the walk stops at the word's end; at p = 1e-3 most words have none."""
    from oracle.philox import faulted_lanes, pauli_code, sample_faults_bernoulli, thresholds
    kinds = ["DEP1", "DEP2", "XERR", "DEP2", "DEP1", "XERR", "DEP2"] * 3
    seed = 0x1234_5678_9ABC
    shots = list(range(0, 3 * 64)) + [64 * 1000 + 5, 64 * 77777 + 63]
    got = sample_faults_bernoulli(seed, kinds, p, shots)
    _, tg = thresholds(p)
    expect = {s: [] for s in shots}
    for w in sorted({s >> 6 for s in shots}):
        for c, kind in enumerate(kinds):
            for lane in faulted_lanes(seed, c, w, tg):
                s = (w << 6) | lane
                if s in expect:
                    expect[s].append((c, pauli_code(seed, c, w, lane, kind)))
    for s in shots:
        assert got[s] == sorted(expect[s]), s
    if p >= 0.05:
        assert max(len(v) for v in got.values()) >= 3
