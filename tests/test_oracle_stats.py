"""Pins of the oracle's statistics (Sec. 4.1, App. C, App. D), CPU only."""
import math
import os

import pytest

from oracle import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table3():
    rows = []
    for line in open(os.path.join(GOLDEN, "loss_table3.txt")):
        t = line.split("#", 1)[0].split()
        if t:
            rows.append((t[0], int(t[1]), [float(v) for v in t[2:]]))
    return rows


@pytest.mark.parametrize("name,m,factors", _table3())
def test_loss_factor_reproduces_table3(name, m, factors):
    """App. C Table 3 from Table 1's M: (1-p_l)^-M, printed to 2 decimals (3 s.f. above 10)."""
    for p_l, printed in zip((1e-4, 5e-4, 1e-3, 2e-3), factors):
        f = stats.loss_factor(m, p_l)
        decimals = len(repr(printed).split(".")[1])
        assert round(f, decimals) == printed, (name, p_l, f, printed)


def test_binomial_weights():
    m, p = 1863, 1e-3
    ws = [stats.bin_w(m, w, p) for w in range(m + 1)]
    assert abs(sum(ws) - 1) < 1e-12
    assert abs(sum(w * b for w, b in enumerate(ws)) - m * p) < 1e-9
    assert abs(stats.bin_w(10, 3, 0.2) - math.comb(10, 3) * 0.2**3 * 0.8**7) < 1e-15
    assert stats.bin_w(5, 0, 0.0) == 1.0 and stats.bin_w(5, 1, 0.0) == 0.0


def test_reweight_and_estimators():
    m, p = 50, 0.01
    counts = {w: (100, 100 - 10 * w, w) for w in range(0, 4)}
    pa, pl = stats.reweight(counts, m, p)
    den = sum(stats.bin_w(m, w, p) * (100 - 10 * w) / 100 for w in range(4))
    num = sum(stats.bin_w(m, w, p) * (100 - 10 * w) / 100 * w / (100 - 10 * w) for w in range(4))
    assert abs(pa - den) < 1e-15 and abs(pl - num / den) < 1e-15
    assert stats.estimators(10, 4, 1) == (0.4, 0.25)


def test_truncation_bound():
    m, p = 1000, 1e-3
    b = stats.truncation_bound(m, 5, p)
    direct = sum(stats.bin_w(m, w, p) for w in range(6, m + 1))
    assert abs(b - direct) < 1e-12


def test_lr_interval_zero_successes():
    """With no successes the upper end solves (1-t)^n = 1/R, about log(R)/n (App. D)."""
    n = 1000
    lo, hi = stats.binomial_lr_interval(0, n)
    assert lo == 0.0
    assert abs(hi - (1 - 100 ** (-1 / n))) < 1e-12
    assert abs(hi - math.log(100) / n) < 1e-4


def test_lr_interval_contains_mle_and_shrinks():
    lo, hi = stats.binomial_lr_interval(30, 100)
    assert lo < 0.3 < hi
    lo2, hi2 = stats.binomial_lr_interval(300, 1000)
    assert hi2 - lo2 < hi - lo
    for th in (lo, hi):
        ll = 30 * math.log(th) + 70 * math.log(1 - th)
        top = 30 * math.log(0.3) + 70 * math.log(0.7)
        assert abs(top - ll - math.log(100)) < 1e-9
