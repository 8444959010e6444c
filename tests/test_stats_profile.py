"""Subset-sampling policy and App. D intervals (CPU only).

The oracle's profile-likelihood interval (a general constrained optimiser on the full rate vector,
Eq. profile) is pinned against what the mathematics fixes: with one bin both functionals reduce to a
single binomial rate, whose likelihood-ratio interval is pinned by its closed form at k = 0
(1 - R^(-1/n)); with two bins the p_acc profile is recomputed by brute force over a fine grid of one
rate (the other follows from the constraint).  The library's interval (per-bin Lagrange conditions)
must then equal the oracle's on random count tables, with and without the d_e rule and known bins.
"""
import math

import numpy as np
import pytest

from oracle import stats as ostats
from paper_2609_19116_b300 import stats as pstats

M, P = 13097, 1e-3


def test_binomial_lr_interval_closed_form_at_zero():
    for n in (10, 137, 5000):
        lo, hi = ostats.binomial_lr_interval(0, n, 100.0)
        assert lo == 0.0
        assert abs(hi - (1 - 100.0 ** (-1.0 / n))) < 1e-12


@pytest.mark.parametrize("n,k", [(150, 140), (80, 3), (40, 0), (60, 60)])
def test_oracle_profile_single_bin_reduces_to_binomial(n, k):
    """One bin: p_acc = B a, so its interval is B times the binomial interval of (k accepted, n)."""
    b = ostats.bin_w(M, 2, P)
    est, lo, hi = ostats.profile_interval({2: (n, k, 0)}, M, P, "p_acc")
    blo, bhi = ostats.binomial_lr_interval(k, n)
    assert abs(est - b * k / n) <= 1e-9 * b  # the optimiser keeps rates within 1e-12 of 0 and 1
    assert abs(lo / b - blo) < 2e-6 and abs(hi / b - bhi) < 2e-6


@pytest.mark.parametrize("acc,err", [(150, 3), (40, 0), (25, 25), (90, 31)])
def test_oracle_profile_single_bin_p_le_reduces_to_binomial(acc, err):
    """One bin: p_le = l, a binomial rate over the accepted shots (the acceptance drops out)."""
    est, lo, hi = ostats.profile_interval({3: (acc + 50, acc, err)}, M, P, "p_le")
    blo, bhi = ostats.binomial_lr_interval(err, acc)
    assert abs(est - err / acc) < 1e-9
    assert abs(lo - blo) < 2e-6 and abs(hi - bhi) < 2e-6


def _grid_profile_two_bins(c1, c2, b1, b2, r=100.0, grid=200001):
    """Brute force: the constrained maximum of l1(a1) + l2(a2) with b1 a1 + b2 a2 = theta, over a fine
    grid of a1 (a2 from the constraint), endpoints by bisection on theta."""
    def ll(k, n, a):
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(k > 0, k * np.log(a), 0.0) + np.where(n - k > 0, (n - k) * np.log1p(-a), 0.0)
    a1 = np.linspace(0.0, 1.0, grid)[1:-1]

    def prof(theta):
        a2 = (theta - b1 * a1) / b2
        ok = (a2 > 0) & (a2 < 1)
        if not ok.any():
            return -np.inf
        return float(np.max(ll(c1[1], c1[0], a1[ok]) + ll(c2[1], c2[0], a2[ok])))
    est = b1 * c1[1] / c1[0] + b2 * c2[1] / c2[0]
    top = ll(c1[1], c1[0], c1[1] / c1[0]) + ll(c2[1], c2[0], c2[1] / c2[0])
    floor = float(top) - math.log(r)

    def bis(a, b):
        for _ in range(60):
            mid = 0.5 * (a + b)
            if prof(mid) >= floor:
                a = mid
            else:
                b = mid
        return 0.5 * (a + b)
    return est, bis(est, 0.0), bis(est, b1 + b2)


def test_oracle_profile_two_bins_matches_grid_brute_force():
    c = {2: (300, 200, 1), 5: (120, 30, 4)}
    est, lo, hi = ostats.profile_interval(c, M, P, "p_acc")
    b1, b2 = ostats.bin_w(M, 2, P), ostats.bin_w(M, 5, P)
    g_est, g_lo, g_hi = _grid_profile_two_bins(c[2], c[5], b1, b2)
    assert abs(est - g_est) <= 1e-12 * est
    assert abs(lo - g_lo) <= 1e-4 * est and abs(hi - g_hi) <= 1e-4 * est


def _random_table(rng, bins=5, d_e=0):
    c = np.zeros((bins, 3), dtype=np.int64)
    for w in range(1, bins):
        n = int(rng.integers(20, 400))
        a = int(rng.binomial(n, rng.uniform(0.05, 0.9)))
        e = 0 if w < d_e else int(rng.binomial(a, rng.uniform(0.0, 0.3)))
        c[w] = (n, a, e)
    return c


@pytest.mark.parametrize("case", range(4))
def test_library_profile_interval_equals_oracle(case):
    rng = np.random.default_rng(100 + case)
    d_e = (0, 2, 0, 3)[case]
    fixed = {0: 1.0} if case % 2 else None
    c = _random_table(rng, bins=5, d_e=d_e)
    cd = {w: tuple(int(v) for v in c[w]) for w in range(len(c)) if c[w, 0] > 0}
    for q in ("p_acc", "p_le"):
        got = pstats.profile_interval(c, M, P, q, d_e=d_e, fixed_accept=fixed)
        est, lo, hi = ostats.profile_interval(cd, M, P, q, d_e=d_e, fixed_accept=fixed)
        scale = max(est, 1e-300)
        assert abs(got["estimate"] - est) <= 1e-9 * scale
        assert abs(got["lo"] - lo) <= 2e-5 * scale, (q, got, lo)
        assert abs(got["hi_stat"] - hi) <= 2e-5 * scale, (q, got, hi)
        assert got["lo"] <= got["estimate"] <= got["hi_stat"]


def test_truncation_systematic_added_upward_only():
    c = np.array([[0, 0, 0], [200, 150, 0], [100, 40, 2]])
    r = pstats.profile_interval(c, M, P, "p_acc")
    b = pstats.truncation_bound(M, 2, P)
    assert b == r["truncation"] and abs(r["hi"] - (r["hi_stat"] + b)) < 1e-15
    rl = pstats.profile_interval(c, M, P, "p_le")
    assert rl["hi"] >= rl["hi_stat"] and rl["lo"] <= rl["estimate"]


def test_unsampled_bins_are_listed():
    c = np.array([[0, 0, 0], [100, 90, 0], [0, 0, 0], [50, 10, 1]])
    assert pstats.profile_interval(c, M, P, "p_acc")["unsampled"] == [2]


def test_schedule_reaches_every_bin_and_follows_bin_w():
    total, w_max = 100000, 6
    plan = pstats.subset_schedule(M, 2e-4, total, w_max, uniform_fraction=0.2, seed=3)
    assert plan.sum() == total and plan[0] == 0
    assert (plan[1:] >= 0.2 * total // w_max).all()
    # the binomial part: proportions of Bin_w(p) conditioned on 1 <= w <= w_max, within 5 sigma
    bw = np.array([ostats.bin_w(M, w, 2e-4) for w in range(1, w_max + 1)])
    prob = bw / bw.sum()
    part = plan[1:] - (0.2 * total // w_max) - np.array([1 if i < (0.2 * total) % w_max else 0
                                                          for i in range(w_max)])
    n = part.sum()
    sig = np.sqrt(n * prob * (1 - prob))
    assert (np.abs(part - n * prob) <= 5 * sig + 1).all()


def test_p_curve_from_one_sample_set_equals_reweighting():
    c = np.array([[50, 50, 0], [200, 150, 0], [100, 40, 2], [60, 10, 3]])
    ps = [1e-4, 5e-4, 1e-3, 2e-3]
    acc, le = pstats.reweight_curve(c, M, ps)
    cd = {w: tuple(int(v) for v in c[w]) for w in range(len(c))}
    for i, p in enumerate(ps):
        oa, ol = ostats.reweight(cd, M, p)
        # the library forms log C(M, w) with lgamma, the oracle by summing integer logs: ~1e-11 apart
        assert abs(acc[i] - oa) <= 1e-9 * oa and abs(le[i] - ol) <= 1e-9 * max(ol, 1e-300)
