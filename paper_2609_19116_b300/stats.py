"""Host-side statistics of subset sampling (Sec. 4.1, App. C, App. D).

Per fault weight w the sampler returns n_w (drawn), n_w^acc (accepted) and n_w^err (accepted and
logically wrong).  The per-weight rates carry no dependence on p, so one set of counts gives the
whole curve (Sec. 4.1):  p_acc = sum_w Bin_w(p) p_acc^(w),  p_acc p_le = sum_w Bin_w(p) p_acc^(w)
p_le^(w),  Bin_w(p) = C(M, w) p^w (1-p)^(M-w).
"""
from __future__ import annotations

import math

import numpy as np


def log_bin_weight(m: int, w: int, p: float) -> float:
    """log Bin_w(p) with log C(M, w) = lgamma(M+1) - lgamma(w+1) - lgamma(M-w+1)."""
    if w < 0 or w > m:
        return -math.inf
    if p <= 0.0:
        return 0.0 if w == 0 else -math.inf
    if p >= 1.0:
        return 0.0 if w == m else -math.inf
    return (math.lgamma(m + 1) - math.lgamma(w + 1) - math.lgamma(m - w + 1)
            + w * math.log(p) + (m - w) * math.log1p(-p))


def bin_weight(m: int, w: int, p: float) -> float:
    return math.exp(log_bin_weight(m, w, p))


def per_weight_rates(counts):
    """counts: array (W, 3) of (n_w, n_w^acc, n_w^err) -> arrays p_acc^(w), p_le^(w) (nan when
    undefined), Eq. estimators."""
    c = np.asarray(counts, dtype=np.float64)
    n, a, e = c[:, 0], c[:, 1], c[:, 2]
    with np.errstate(invalid="ignore", divide="ignore"):
        pa = np.where(n > 0, a / np.where(n > 0, n, 1), np.nan)
        pl = np.where(a > 0, e / np.where(a > 0, a, 1), np.nan)
    return pa, pl


def reweight(counts, m: int, p: float):
    """(p_acc, p_le) at rate p from per-weight counts (Eq. reweight); bins never drawn are left out
    (their mass is reported by `truncation_bound`)."""
    pa, pl = per_weight_rates(counts)
    num = den = 0.0
    for w in range(len(pa)):
        if np.isnan(pa[w]):
            continue
        b = bin_weight(m, w, p)
        den += b * pa[w]
        if not np.isnan(pl[w]):
            num += b * pa[w] * pl[w]
    return den, (num / den if den > 0 else float("nan"))


def truncation_bound(m: int, w_max: int, p: float) -> float:
    """B = sum_{w > w_max} Bin_w(p): the most the unsampled weights can add (App. D)."""
    if p <= 0.0:
        return 0.0
    # complement of the binomial CDF, summed over the (few) bins up to w_max
    return max(0.0, 1.0 - sum(bin_weight(m, w, p) for w in range(0, min(w_max, m) + 1)))


def likelihood_interval(k: int, n: int, r: float = 100.0):
    """Values of a binomial proportion whose likelihood is within a factor r of the maximum
    (App. D uses r = 100), endpoints by bisection."""
    if n <= 0:
        return 0.0, 1.0

    def ll(t):
        out = 0.0
        if k:
            out += k * math.log(t) if t > 0 else -math.inf
        if n - k:
            out += (n - k) * math.log(1 - t) if t < 1 else -math.inf
        return out

    hat = k / n
    floor = ll(hat) - math.log(r)

    def edge(inside, outside):
        for _ in range(100):
            mid = 0.5 * (inside + outside)
            if ll(mid) >= floor:
                inside = mid
            else:
                outside = mid
        return 0.5 * (inside + outside)

    lo = 0.0 if ll(0.0) >= floor else edge(hat, 0.0)
    hi = 1.0 if ll(1.0) >= floor else edge(hat, 1.0)
    return lo, hi


def loss_factor(m: int, p_loss: float) -> float:
    """Factor on the expected attempts from M independent, detected loss channels: (1-p_l)^-M
    (App. C)."""
    return math.exp(-m * math.log1p(-p_loss))
