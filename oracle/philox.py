"""Philox4x32-10 and the random-number contract, oracle side (test infrastructure only).

The paper does not fix a random number generator.  The sampled quantities are the ones it
defines: per shot, each noise channel independently resolves to a non-identity Pauli with
probability p, uniformly among the 4^k-1 strings (Sec. 4), the number of such channels being the
fault weight w; measurement outcomes follow the Born rule.  The contract below makes those draws
reproducible bit for bit from (seed, shot index); the CUDA library implements the same contract
in its own code.

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (c0,c1,c2,c3), key (k0,k1), ten rounds
of  (c0,c1,c2,c3) <- (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)),  with the key
bumped by the Weyl constants between rounds.  key = (seed mod 2^32, seed >> 32).

Contract (c3 is the stream tag; shots are grouped in 64-shot words w = shot >> 6, lane = shot & 63):
  thresholds   T1 = floor(p * 2^32);  y = 1 - T1/2^32 (exact);  for s = 0..63, with y_s = y^(s+1)
               formed by s successive FP64 multiplications, TG[s] = floor((1 - y_s) * 2^32).
  TAG_WORD 0   u = philox(c >> 2, w, 0, 0)[c & 3]:  the first faulted lane of channel c in word w is
               the smallest s with u < TG[s]; none if u >= TG[63].
  TAG_SKIP 1   the k-th further draw d_k = philox(c, w, k >> 2, 1)[k & 3] gives a skip s (smallest
               s with d_k < TG[s], none -> stop); the next faulted lane is previous + 1 + s (< 64).
               Lanes are therefore independent Bernoulli(T1/2^32) (geometric gaps).
  TAG_PAULI 2  for a faulted lane j: x = philox(c, w, j, 2)[0]; code = 1 + ((x * z) >> 32) with
               z = 3 (one-qubit channel) or 15 (two-qubit channel); XERR channels are always X.
               Two-qubit code i means (P_a, P_b) = (i >> 2, i & 3) with 0=I,1=X,2=Y,3=Z.
  TAG_MEAS 3   readout k of shot s: x = philox(k, s mod 2^32, s >> 32, 3);
               u = ((x0 >> 5) * 2^26 + (x1 >> 6)) / 2^53;  outcome 1 iff u < p1 (FP64).
  TAG_EXACT 4  exact-weight mode (fault weight fixed to w): Floyd's algorithm picks w distinct
               channels; draw i of shot s is philox(i, s mod 2^32, s >> 32, 4)[0] and is turned
               into an integer in [0, j] by Lemire's multiply-shift with rejection.  The Pauli of a
               chosen channel c is drawn from philox(c, s mod 2^32, s >> 32, 5)[0] as above.
"""
from __future__ import annotations

import numpy as np

MASK = np.uint64(0xFFFFFFFF)
M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
TAG_WORD, TAG_SKIP, TAG_PAULI, TAG_MEAS, TAG_EXACT, TAG_EXACT_PAULI = 0, 1, 2, 3, 4, 5


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit values held in uint64 (Salmon et al. 2011)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & MASK)
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)


def thresholds(p: float):
    """(T1, TG[0..63]) of the contract; FP64 operations in the stated order."""
    if not (0.0 <= p < 1.0):
        raise ValueError("p must lie in [0, 1)")
    t1 = int(np.floor(p * 4294967296.0))
    t1 = min(t1, 0xFFFFFFFF)
    y = 1.0 - t1 / 4294967296.0
    tg = []
    ys = y
    for _ in range(64):
        tg.append(min(int(np.floor((1.0 - ys) * 4294967296.0)), 0xFFFFFFFF))
        ys = ys * y
    return t1, np.array(tg, dtype=np.uint64)


def _first_below(u: int, tg) -> int:
    """Smallest s with u < tg[s], or 64 when there is none."""
    for s in range(64):
        if u < int(tg[s]):
            return s
    return 64


def faulted_lanes(seed: int, c: int, w: int, tg) -> list:
    """Faulted lanes of channel c in word w (TAG_WORD then TAG_SKIP draws)."""
    k0, k1 = key_of(seed)
    x = philox4x32_10(c >> 2, w, 0, TAG_WORD, k0, k1)
    u = int(x[c & 3])
    lane = _first_below(u, tg)
    if lane >= 64:
        return []
    lanes = [lane]
    k = 0
    while True:
        d = philox4x32_10(c, w, k >> 2, TAG_SKIP, k0, k1)
        s = _first_below(int(d[k & 3]), tg)
        k += 1
        if s >= 64:
            break
        lane = lane + 1 + s
        if lane >= 64:
            break
        lanes.append(lane)
    return lanes


def pauli_code(seed: int, c: int, w: int, lane: int, kind: str) -> int:
    if kind == "XERR":
        return 1
    z = 15 if kind == "DEP2" else 3
    k0, k1 = key_of(seed)
    x = int(philox4x32_10(c, w, lane, TAG_PAULI, k0, k1)[0])
    return 1 + ((x * z) >> 32)


def word_events(seed: int, n_channels: int, words, tg):
    """Boolean (n_channels, len(words)) array: does channel c fault anywhere in word w.

    Vectorised TAG_WORD draws; used to find the rare (channel, word) pairs that need lanes."""
    k0, k1 = key_of(seed)
    words = np.asarray(words, dtype=np.uint64)
    groups = np.arange((n_channels + 3) // 4, dtype=np.uint64)
    G, Wd = np.meshgrid(groups, words, indexing="ij")
    x = philox4x32_10(G, Wd, 0, TAG_WORD, k0, k1)
    u = np.stack(x, axis=1).reshape(len(groups) * 4, len(words))[:n_channels]
    return u < tg[63]


def first_below_vec(u, tg):
    """Vectorised: smallest s with u < tg[s], or 64."""
    return np.searchsorted(tg, u, side="right")


def sample_faults_bernoulli(seed: int, channel_kinds, p: float, shots):
    """Per shot: sorted list of (channel, pauli code) under independent Bernoulli(p) channels.

    Follows Sec. 4: every channel independently resolves to a non-identity Pauli with probability
    p (quantised to T1/2^32 by the contract), uniformly among the 4^k-1 strings.  The draws are
    those of `faulted_lanes` and `pauli_code`, evaluated for all (channel, word) events at once."""
    shots = [int(s) for s in shots]
    _, tg = thresholds(p)
    words = sorted({s >> 6 for s in shots})
    out = {s: [] for s in shots}
    if not words or not channel_kinds:
        return out
    k0, k1 = key_of(seed)
    wanted = {}
    for s in shots:
        wanted.setdefault(s >> 6, set()).add(s & 63)
    # word-level draws, in blocks of words to bound memory
    ev_c, ev_w, ev_u = [], [], []
    groups = np.arange((len(channel_kinds) + 3) // 4, dtype=np.uint64)
    for b in range(0, len(words), 256):
        wb = np.array(words[b:b + 256], dtype=np.uint64)
        G, Wd = np.meshgrid(groups, wb, indexing="ij")
        x = philox4x32_10(G, Wd, 0, TAG_WORD, k0, k1)
        u = np.stack(x, axis=1).reshape(len(groups) * 4, len(wb))[:len(channel_kinds)]
        ci, wi = np.nonzero(u < tg[63])
        ev_c.append(ci.astype(np.uint64))
        ev_w.append(wb[wi])
        ev_u.append(u[ci, wi])
    ev_c = np.concatenate(ev_c)
    ev_w = np.concatenate(ev_w)
    lane = first_below_vec(np.concatenate(ev_u), tg).astype(np.int64)
    pairs = [(ev_c, ev_w, lane.copy())]
    active = np.ones(len(lane), dtype=bool)
    k = 0
    while active.any():
        idx = np.nonzero(active)[0]
        d = philox4x32_10(ev_c[idx], ev_w[idx], k >> 2, TAG_SKIP, k0, k1)[k & 3]
        s = first_below_vec(d, tg).astype(np.int64)
        nl = lane[idx] + 1 + s
        ok = (s < 64) & (nl < 64)
        lane[idx[ok]] = nl[ok]
        active[idx[~ok]] = False
        pairs.append((ev_c[idx[ok]], ev_w[idx[ok]], nl[ok]))
        k += 1
    C = np.concatenate([pp[0] for pp in pairs])
    Wv = np.concatenate([pp[1] for pp in pairs])
    Lv = np.concatenate([pp[2] for pp in pairs])
    keep = np.array([int(l) in wanted[int(w)] for w, l in zip(Wv, Lv)], dtype=bool)
    C, Wv, Lv = C[keep], Wv[keep], Lv[keep]
    xs = philox4x32_10(C, Wv, Lv.astype(np.uint64), TAG_PAULI, k0, k1)[0]
    for c, w, l, x in zip(C.tolist(), Wv.tolist(), Lv.tolist(), xs.tolist()):
        kind = channel_kinds[c]
        if kind == "XERR":
            code = 1
        else:
            z = 15 if kind == "DEP2" else 3
            code = 1 + ((int(x) * z) >> 32)
        out[(w << 6) | l].append((c, code))
    for s in out:
        out[s].sort()
    return out


def _bounded(seed: int, shot: int, draw: int, bound: int):
    """Integer in [0, bound) from the TAG_EXACT stream (Lemire's method with rejection)."""
    k0, k1 = key_of(seed)
    lo, hi = shot & 0xFFFFFFFF, shot >> 32
    thresh = ((1 << 32) - bound) % bound
    while True:
        x = int(philox4x32_10(draw, lo, hi, TAG_EXACT, k0, k1)[0])
        draw += 1
        m = x * bound
        if (m & 0xFFFFFFFF) >= thresh:
            return m >> 32, draw


def sample_faults_exact(seed: int, channel_kinds, weight: int, shot: int):
    """Exactly `weight` distinct channels, uniformly (Floyd's algorithm), each with a uniform
    non-identity Pauli: the fixed-weight subsets of subset sampling (Sec. 4.1)."""
    m = len(channel_kinds)
    if weight > m:
        raise ValueError("fault weight exceeds the number of channels")
    chosen = set()
    draw = 0
    for j in range(m - weight, m):
        t, draw = _bounded(seed, shot, draw, j + 1)
        chosen.add(j if t in chosen else t)
    k0, k1 = key_of(seed)
    faults = []
    for c in sorted(chosen):
        kind = channel_kinds[c]
        if kind == "XERR":
            code = 1
        else:
            z = 15 if kind == "DEP2" else 3
            x = int(philox4x32_10(c, shot & 0xFFFFFFFF, shot >> 32, TAG_EXACT_PAULI, k0, k1)[0])
            code = 1 + ((x * z) >> 32)
        faults.append((c, code))
    return faults


def readout_uniform(seed: int, k: int, shot: int) -> float:
    """53-bit uniform in [0, 1) for readout k of a shot (TAG_MEAS)."""
    k0, k1 = key_of(seed)
    x = philox4x32_10(k, shot & 0xFFFFFFFF, shot >> 32, TAG_MEAS, k0, k1)
    u53 = (int(x[0]) >> 5) * (1 << 26) + (int(x[1]) >> 6)
    return u53 / 9007199254740992.0
