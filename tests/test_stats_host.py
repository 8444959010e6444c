"""The package's host statistics against the oracle's (independent code) and the paper's Table 3."""
import math
import os

import numpy as np
import pytest

from oracle import stats as ost
from paper_2609_19116_b300 import stats as pst

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_binomial_weights_agree():
    for m, w, p in [(1863, 0, 1e-3), (1863, 5, 1e-3), (243, 3, 2e-3), (50, 50, 0.3), (10, 3, 0.0)]:
        assert math.isclose(pst.bin_weight(m, w, p), ost.bin_w(m, w, p), rel_tol=1e-10, abs_tol=1e-300)  # lgamma vs sums of logs: ~M eps in the exponent


def test_reweight_agrees_with_oracle():
    rng = np.random.default_rng(0)
    counts = np.zeros((8, 3), dtype=np.int64)
    for w in range(8):
        n = int(rng.integers(50, 500))
        a = int(rng.integers(0, n + 1))
        e = int(rng.integers(0, a + 1))
        counts[w] = (n, a, e)
    counts[6] = (0, 0, 0)  # a bin never drawn
    for p in (5e-4, 1e-3, 2e-3):
        a1, l1 = pst.reweight(counts, 1500, p)
        a2, l2 = ost.reweight({w: tuple(int(v) for v in counts[w]) for w in range(8)}, 1500, p)
        assert math.isclose(a1, a2, rel_tol=1e-10) and math.isclose(l1, l2, rel_tol=1e-10)


def test_truncation_and_intervals_agree():
    assert math.isclose(pst.truncation_bound(1000, 5, 1e-3), ost.truncation_bound(1000, 5, 1e-3), rel_tol=1e-9)
    for k, n in [(0, 1000), (3, 100), (50, 100), (100, 100)]:
        a, b = pst.likelihood_interval(k, n), ost.binomial_lr_interval(k, n)
        assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] - b[1]) < 1e-12


def _table3():
    for line in open(os.path.join(GOLDEN, "loss_table3.txt")):
        t = line.split("#", 1)[0].split()
        if t:
            yield t[0], int(t[1]), [float(v) for v in t[2:]]


@pytest.mark.parametrize("name,m,factors", list(_table3()))
def test_loss_factor_table3(name, m, factors):
    for p_l, printed in zip((1e-4, 5e-4, 1e-3, 2e-3), factors):
        decimals = len(repr(printed).split(".")[1])
        assert round(pst.loss_factor(m, p_l), decimals) == printed
