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


def subset_loglik(counts: dict, a: dict, l: dict) -> float:
    """Joint log-likelihood of the per-bin rates (App. D, Eq. loglik-split): per bin w, a binomial term
    for the n_w^acc accepted of n_w shots at rate a_w plus a binomial term for the n_w^err failures of
    the accepted at rate l_w; bins are independent, so the terms add."""
    out = 0.0
    for w, (n, n_acc, n_err) in counts.items():
        out += _binom_loglik(n_acc, n, a[w])
        if n_acc:
            out += _binom_loglik(n_err, n_acc, l[w])
    return out


def profile_interval(counts: dict, m: int, p: float, quantity: str, r: float = 100.0, d_e: int = 0,
                     fixed_accept=None):
    """Likelihood-ratio interval of a reweighted rate (App. D, Eq. profile), computed plainly: for a
    candidate theta, the log-likelihood of Eq. loglik-split is maximised over every free bin rate
    (a_w, and l_w for w >= d_e) subject to f(rates) = theta by a general constrained optimiser
    (scipy SLSQP); theta is kept while that maximum is within log r of the unconstrained maximum, and
    the endpoints are found by bisection.  f = sum_w Bin_w(p) a_w (p_acc) or its ratio with
    sum_w Bin_w(p) a_w l_w (p_le, Eq. reweight).  Bins w < d_e have l_w = 0; fixed_accept = {w: a}
    holds known acceptances.  Only bins with n_w > 0 carry free rates.  No systematic is added."""
    import numpy as np
    from scipy.optimize import minimize

    fixed_accept = dict(fixed_accept or {})
    bins = sorted(w for w, (n, _, _) in counts.items() if n > 0 and w not in fixed_accept)
    B = {w: bin_w(m, w, p) for w in list(bins) + list(fixed_accept)}
    free_l = [w for w in bins if w >= d_e and counts[w][1] > 0]
    eps = 1e-12

    def unpack(v):
        a = {w: v[i] for i, w in enumerate(bins)}
        l = {w: 0.0 for w in bins}
        for j, w in enumerate(free_l):
            l[w] = v[len(bins) + j]
        return a, l

    def f(v):
        a, l = unpack(v)
        den = sum(B[w] * a[w] for w in bins) + sum(B[w] * x for w, x in fixed_accept.items())
        if quantity == "p_acc":
            return den
        return sum(B[w] * a[w] * l[w] for w in bins) / den

    def neg_ll(v):
        a, l = unpack(v)
        return -subset_loglik({w: counts[w] for w in bins}, a, l)

    mle = [min(max(counts[w][1] / counts[w][0], eps), 1 - eps) for w in bins]
    mle += [min(max(counts[w][2] / counts[w][1], eps), 1 - eps) for w in free_l]
    bounds = [(eps, 1 - eps)] * len(mle)
    top = -neg_ll(np.array(mle))
    est = f(np.array(mle))

    def constrained_max(theta):
        best = -math.inf
        for start in (mle, [0.5] * len(mle)):
            res = minimize(neg_ll, np.array(start), method="SLSQP", bounds=bounds,
                           constraints=[{"type": "eq", "fun": lambda v: f(v) - theta}],
                           options={"ftol": 1e-14, "maxiter": 1000})
            if res.success and abs(f(res.x) - theta) < 1e-9 * max(1.0, abs(theta)):
                best = max(best, -res.fun)
        return best

    def inside(theta):
        return constrained_max(theta) >= top - math.log(r)

    def bisect(a, b):  # a inside, b outside
        for _ in range(60):
            mid = 0.5 * (a + b)
            if inside(mid):
                a = mid
            else:
                b = mid
        return 0.5 * (a + b)

    lo_end = 0.0 if quantity == "p_le" else sum(B[w] * x for w, x in fixed_accept.items())
    hi_end = 1.0 if quantity == "p_le" else lo_end + sum(B[w] for w in bins)
    lo = lo_end if inside(lo_end + 1e-12 * max(est, 1e-300)) else bisect(est, lo_end)
    hi = hi_end if inside(hi_end * (1 - 1e-12)) else bisect(est, hi_end)
    return est, lo, hi
