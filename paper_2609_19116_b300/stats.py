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


# ---- subset-sampling schedule and p-curve reuse (Sec. 4.1) ------------------------------------------

def subset_schedule(m: int, p: float, total: int, w_max: int, *, uniform_fraction: float = 0.1,
                    skip_zero: bool = True, seed: int = 0) -> np.ndarray:
    """Shots per fault weight w = 0..w_max (Sec. 4.1): a fraction 1 - uniform_fraction of `total` drawn
    from Bin_w(p) (which reproduces physical sampling), truncated at w_max, and the rest spread evenly
    over w = 1..w_max so that every bin up to w_max is reached.  With skip_zero the weight-0 bin, whose
    rates are known (every noiseless shot is accepted and correct), gets no shots and the Bin_w draw
    is conditioned on w >= 1."""
    if w_max < 1 or total < 0 or not (0.0 <= uniform_fraction <= 1.0):
        raise ValueError("need w_max >= 1, total >= 0 and uniform_fraction in [0, 1]")
    w0 = 1 if skip_zero else 0
    lw = np.array([log_bin_weight(m, w, p) for w in range(w0, w_max + 1)])
    prob = np.exp(lw - lw.max())
    prob /= prob.sum()
    n_uni = int(round(uniform_fraction * total))
    rng = np.random.default_rng(seed)
    out = np.zeros(w_max + 1, dtype=np.int64)
    out[w0:] += rng.multinomial(total - n_uni, prob)
    out[1:] += n_uni // w_max
    out[1:1 + n_uni % w_max] += 1
    return out


def reweight_curve(counts, m: int, ps, *, d_e: int = 0, fixed_accept=None):
    """p_acc(p) and p_le(p) for every p in ps from one set of per-weight counts (Sec. 4.1: the per-bin
    rates carry no p dependence, so one sample set gives the whole curve; the points are correlated).
    Bins w < d_e have p_le^(w) = 0 imposed; fixed_accept = {w: p_acc^(w)} gives known acceptances
    (e.g. {0: 1.0} when the weight-0 bin is not sampled)."""
    pa, pl = per_weight_rates(counts)
    fixed_accept = fixed_accept or {}
    for w, a in fixed_accept.items():
        pa[w] = a
        pl[w] = 0.0
    pl[:min(d_e, len(pl))] = 0.0
    acc, le = [], []
    for p in np.atleast_1d(ps):
        b = np.array([bin_weight(m, w, float(p)) for w in range(len(pa))])
        ok = ~np.isnan(pa)
        den = float(np.sum(b[ok] * pa[ok]))
        ok2 = ok & ~np.isnan(pl)
        num = float(np.sum(b[ok2] * pa[ok2] * pl[ok2]))
        acc.append(den)
        le.append(num / den if den > 0 else float("nan"))
    return np.array(acc), np.array(le)


# ---- profile-likelihood intervals of the reweighted rates (App. D) ------------------------------------
#
# A bin's three outcomes (rejected, accepted and correct, accepted and wrong) have probabilities
# x = (r, c, e) = (1 - a, a (1 - l), a l), a = p_acc^(w), l = p_le^(w); its log-likelihood is
# sum_i n_i log x_i (Eq. loglik-split, the two binomial terms, written in the multinomial form).  Both
# functionals are linear in x at a fixed candidate value: p_acc = sum_w B_w (c_w + e_w) and, for
# p_le = N / D, N - theta D = sum_w B_w (e_w (1 - theta) - theta c_w).  The constrained maximum of
# Eq. profile is then a concave problem whose Lagrange conditions decouple per bin: for a multiplier
# mu each bin maximises sum_i n_i log x_i + g . x on the simplex, g = mu x (the functional's
# coefficients), solved by x_i = n_i / (nu - g_i) with sum x = 1 (one root per bin); a component with
# no counts takes the remaining mass only when its coefficient exceeds nu.

def _bin_argmax(n, g):
    """Per bin (rows): argmax of sum_i n_i log x_i + sum_i g_i x_i over the probability simplex.

    nu solves f(nu) = sum_{n_i > 0} n_i / (nu - g_i) - 1 = 0 above max g_i; f is convex and decreasing
    there, so Newton's method started left of the root (at max g_i + its count, where f >= 0) rises
    monotonically to it."""
    n = np.asarray(n, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    pos = n > 0
    gs = np.where(pos, g, -np.inf)
    k = np.argmax(gs, axis=1)
    rows = np.arange(len(n))
    nu = gs[rows, k] + n[rows, k]
    for _ in range(100):
        with np.errstate(divide="ignore", invalid="ignore"):
            d = np.where(pos, nu[:, None] - g, 1.0)
            f = np.where(pos, n / d, 0.0).sum(axis=1) - 1.0
            fp = np.where(pos, n / (d * d), 0.0).sum(axis=1)
        step = f / fp
        nu = nu + step
        if np.all(np.abs(step) <= 1e-15 * np.maximum(1.0, np.abs(nu))):
            break
    gz = np.where(~pos, g, -np.inf).max(axis=1)
    take = gz > nu
    nu = np.where(take, gz, nu)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = np.where(pos, n / (nu[:, None] - g), 0.0)
    rest = np.clip(1.0 - x.sum(axis=1), 0.0, None)
    zidx = np.argmax(np.where(~pos, g, -np.inf), axis=1)
    x[rows, zidx] += np.where(take, rest, 0.0)
    return x / x.sum(axis=1, keepdims=True)


def _loglik(n, x):
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(n > 0, n * np.log(np.where(x > 0, x, 1.0)), 0.0)
        t = np.where((n > 0) & (x <= 0), -np.inf, t)
    return float(t.sum())


def _root(f, a, b):
    """Root of f between a and b (opposite signs) by Brent's method."""
    from scipy.optimize import brentq
    return brentq(f, a, b, xtol=1e-300, rtol=1e-15, maxiter=500)


def _expand(f, start, sign):
    """Walk start * 2^k (k = 0, 1, ...) in the direction `sign` until f changes sign from f(0)."""
    x = sign * start
    while abs(x) < 1e290:
        if f(x) < 0:
            return x
        x *= 2.0
    return None


def profile_interval(counts, m: int, p: float, quantity: str = "p_le", *, r: float = 100.0, d_e: int = 0,
                     fixed_accept=None, w_max: int | None = None):
    """Likelihood-ratio interval of the reweighted p_acc or p_le at rate p (App. D, Eq. profile): the
    values theta whose constrained maximum of the joint log-likelihood sum_w l_w (Eq. loglik-split)
    stays within log r of the overall maximum.  Bins w < d_e have p_le^(w) = 0 imposed (their accepted
    shots must all be correct); fixed_accept = {w: a} fixes known acceptances; bins never sampled
    (n_w = 0) are absent and listed.  The truncation systematic B = sum_{w > w_max} Bin_w(p) (w_max =
    the last bin by default) is added to the upper endpoint only: as B for p_acc and as B / p_acc for
    p_le (the omitted mass in the numerator over the estimated acceptance).
    Returns dict(estimate, lo, hi, truncation, unsampled)."""
    c = np.asarray(counts, dtype=np.int64)
    W = len(c)
    w_max = W - 1 if w_max is None else w_max
    fixed_accept = dict(fixed_accept or {})
    bw = np.array([bin_weight(m, w, p) for w in range(W)])
    sampled = [w for w in range(W) if c[w, 0] > 0 and w not in fixed_accept]
    unsampled = [w for w in range(1, w_max + 1) if c[w, 0] == 0 and w not in fixed_accept]
    for w in sampled:
        if w < d_e and c[w, 2] > 0:
            raise ValueError(f"bin {w} < d_e has logical errors")
    n = np.array([[c[w, 0] - c[w, 1], c[w, 1] - c[w, 2], c[w, 2]] for w in sampled], dtype=np.float64)
    n = n.reshape(-1, 3)
    B = bw[sampled] if sampled else np.zeros(0)
    low = np.array([w < d_e for w in sampled], dtype=bool)
    d_fix = float(sum(bw[w] * a for w, a in fixed_accept.items()))  # known acceptances, no errors
    trunc = truncation_bound(m, w_max, p)
    scale = 1.0 / max(float(B.max()) if len(B) else 1.0, 1e-300)

    def solve(gc, ge):
        """Per-bin maximiser; a bin below d_e keeps e = 0 (a hugely negative coefficient, no counts)."""
        g = np.stack([np.zeros(len(B)), gc, np.where(low, -1e300, ge)], axis=1)
        return _bin_argmax(n, g)

    x0 = solve(np.zeros(len(B)), np.zeros(len(B)))
    l_max = _loglik(n, x0)
    logr = math.log(r)
    acc_hat = d_fix + float(np.sum(B * (x0[:, 1] + x0[:, 2])))
    if quantity == "p_acc":
        # mu > 0 lowers the acceptance of every bin, mu < 0 raises it; theta(mu) is monotone
        def at(mu):
            x = solve(-mu * B, -mu * B)
            return l_max - _loglik(n, x), d_fix + float(np.sum(B * (x[:, 1] + x[:, 2])))

        def edge(sign):
            far = _expand(lambda mu: logr - at(mu)[0], scale, sign)
            if far is None:  # the likelihood never drops by log r: the range's end
                return at(sign * 1e290)[1]
            return at(_root(lambda mu: logr - at(mu)[0], 0.0, far))[1]
        hi = edge(-1.0)
        return {"estimate": acc_hat, "lo": edge(+1.0), "hi": hi + trunc, "hi_stat": hi, "truncation": trunc,
                "unsampled": unsampled}
    if quantity != "p_le":
        raise ValueError("quantity must be 'p_acc' or 'p_le'")
    est = float(np.sum(B * x0[:, 2])) / acc_hat if acc_hat > 0 else float("nan")

    def profile(theta):
        """Constrained maximum of the log-likelihood with p_le = theta: the multiplier mu solves
        sum_w B_w (e_w (1 - theta) - theta c_w) = theta d_fix, whose left side falls as mu grows."""
        def h(mu):
            x = solve(mu * B * theta, -mu * B * (1.0 - theta))
            return float(np.sum(B * (x[:, 2] * (1.0 - theta) - theta * x[:, 1]))) - theta * d_fix
        if h(0.0) >= 0:
            a, b = 0.0, _expand(lambda mu: h(mu), scale, +1.0)
        else:
            a, b = _expand(lambda mu: -h(mu), scale, -1.0), 0.0
        if a is None or b is None:
            return -math.inf
        mu = _root(h, a, b) if h(a) * h(b) < 0 else (a if h(a) == 0 else b)
        x = solve(mu * B * theta, -mu * B * (1.0 - theta))
        return _loglik(n, x)

    def inside(theta):
        return profile(theta) - (l_max - logr)

    if not np.isfinite(est) or len(B) == 0:
        return {"estimate": est, "lo": 0.0, "hi": 1.0, "hi_stat": 1.0, "truncation": trunc, "unsampled": unsampled}
    tiny, top = 1e-300, 1.0 - 1e-12
    lo = 0.0 if inside(tiny) >= 0 else _root(inside, tiny, est)
    hi = 1.0 if inside(top) >= 0 else _root(inside, est, top)
    return {"estimate": est, "lo": lo, "hi": min(1.0, hi + (trunc / acc_hat if acc_hat > 0 else 0.0)),
            "hi_stat": hi, "truncation": trunc, "unsampled": unsampled}


# ---- subset sampling on the device (Sec. 4.1) ---------------------------------------------------------

def sample_subsets(circ, plan, *, seed: int, chi_max: int, cutoff: float, precision: int = 0, shot0: int = 0,
                   w_stride: int = 1 << 36):
    """Per-weight counts (n_w, n_w^acc, n_w^err) from plan[w] shots with exactly w faults each (channels
    drawn uniformly, Sec. 4.1): the fixed-weight pre-screen over plan[w] drawn shots (its rejections
    count as rejected), then the MPS engine on its survivors.  Weight w uses the shot range starting at
    shot0 + w * w_stride, so the bins are independent.  Counts carry no p dependence: evaluate them at
    any p with reweight_curve / profile_interval."""
    from . import api
    plan = np.asarray(plan, dtype=np.int64)
    out = np.zeros((len(plan), 3), dtype=np.uint64)
    for w, nw in enumerate(plan):
        if nw <= 0:
            continue
        base = shot0 + w * w_stride
        pre = api.pauli_prescreen(circ, base, int(nw), p=0.0, seed=seed, fault_weight=w, w_max=63)
        out[w, 0] = nw
        if pre["n_kept"] == 0:
            continue
        counts, _ = api.mps_sample_batch(circ, pre["survivors"], p=0.0, seed=seed, chi_max=chi_max, cutoff=cutoff,
                                         precision=precision, fault_weight=w, w_max=63, per_shot=False)
        out[w, 1] = counts[:, 1].sum()
        out[w, 2] = counts[:, 2].sum()
    return out
