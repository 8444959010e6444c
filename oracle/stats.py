"""Subset-sampling statistics (Sec. 4.1, App. C, App. D), test infrastructure only.

Exact binomial weights are formed in log space from sums of logarithms of integers.
"""
from __future__ import annotations

import math


def log_binom(m: int, w: int) -> float:
    """log C(m, w) as a sum of logs of integers."""
    if w < 0 or w > m:
        return -math.inf
    w = min(w, m - w)
    return sum(math.log(m - w + i) - math.log(i) for i in range(1, w + 1))


def bin_w(m: int, w: int, p: float) -> float:
    """Bin_w(p) = C(M, w) p^w (1-p)^(M-w): probability that exactly w channels fire (Sec. 4.1)."""
    if p == 0.0:
        return 1.0 if w == 0 else 0.0
    return math.exp(log_binom(m, w) + w * math.log(p) + (m - w) * math.log1p(-p))


def estimators(n: int, n_acc: int, n_err: int):
    """Per-bin estimates (Eq. estimators): p_acc^(w) = n_acc/n, p_le^(w) = n_err/n_acc."""
    pa = n_acc / n if n else float("nan")
    pl = n_err / n_acc if n_acc else float("nan")
    return pa, pl


def reweight(counts: dict, m: int, p: float):
    """(p_acc, p_le) from per-weight counts {w: (n, n_acc, n_err)} (Eq. reweight).

    Bins with n = 0 contribute nothing; bins with n_acc = 0 contribute nothing to the numerator."""
    num = 0.0
    den = 0.0
    for w, (n, n_acc, n_err) in counts.items():
        if n == 0:
            continue
        b = bin_w(m, w, p)
        pa, pl = estimators(n, n_acc, n_err)
        den += b * pa
        if n_acc:
            num += b * pa * pl
    return den, (num / den if den > 0 else float("nan"))


def truncation_bound(m: int, w_max: int, p: float) -> float:
    """B = sum_{w > w_max} Bin_w(p) (App. D, truncation systematic)."""
    return max(0.0, 1.0 - sum(bin_w(m, w, p) for w in range(0, w_max + 1)))


def loss_factor(m: int, p_l: float) -> float:
    """Multiplicative factor on the expected attempts from M independent loss channels, (1-p_l)^-M
    (App. C)."""
    return (1.0 - p_l) ** (-m)


def _binom_loglik(k: int, n: int, th: float) -> float:
    out = 0.0
    if k:
        out += k * math.log(th) if th > 0 else -math.inf
    if n - k:
        out += (n - k) * math.log1p(-th) if th < 1 else -math.inf
    return out


def binomial_lr_interval(k: int, n: int, r: float = 100.0):
    """Likelihood-ratio interval of a binomial proportion: the values whose likelihood is within a
    factor R of the maximum (App. D, R = 100), endpoints by bisection."""
    if n == 0:
        return 0.0, 1.0
    mle = k / n
    top = _binom_loglik(k, n, mle)
    thr = top - math.log(r)

    def inside(th):
        return _binom_loglik(k, n, th) >= thr

    def bisect(a, b):  # a inside, b outside
        for _ in range(200):
            mid = 0.5 * (a + b)
            if inside(mid):
                a = mid
            else:
                b = mid
        return 0.5 * (a + b)

    lo = 0.0 if inside(0.0) else bisect(mle, 0.0)
    hi = 1.0 if inside(1.0) else bisect(mle, 1.0)
    return lo, hi
