"""The approximate counter CountingProVe_SLR, FP64 (test infrastructure only).

Sec. 2.3 describes the approximation of CountingProVe: the property's domain
is split again and again while a sample of violation points is kept evenly
balanced between the two halves, one half is followed at each split, and only
the final leaf is counted exactly; that count, scaled by 2^s for s splits,
estimates the whole domain's.  Sec. 4 (Table 1) uses it with the exact counter
of Alg. 1 (this package's ``counter.count``) as the backend on the leaf and
reports a lower bound of the violation rate with confidence above 99 %.

Steps of one trial, as written here (each reading is listed in the design notes):

  1. Start from the root box [a, b].
  2. For split j = 0 .. s - 1:
     a. take the widest side of the current box (float64 widths of the
        float32 endpoints, ties to the lowest index);
     b. sample n points uniformly in the box, x = lo + (hi - lo) u, with u
        drawn by SplitMix64 (below) and the arithmetic in float64 without
        fused multiply-add;
     c. classify each point with a float64 forward pass (``slr.unsafe_points``);
     d. the split point is the lower median of the unsafe points' coordinates
        on that side (the midpoint when no sampled point is unsafe), rounded to
        the nearest float32; when it is not strictly inside the side, the
        float32 midpoint; when that is not inside either, stop splitting;
     e. a fair coin (one SplitMix64 draw) keeps the lower or the upper half.
  3. Count the leaf exactly to depth D_leaf: [lo_l, hi_l] in units of 2^-D_leaf
     of the leaf's volume.
  4. Estimate the violation rate as X = 2^s lo_l 2^-D_leaf vol(leaf)/vol(root).

Guarantee (derived here, not printed in the paper).  Whatever the split
points, the coin picks each half with probability 1/2, so E[2 c(half)] =
c(parent) for the unsafe volume c; by induction E[2^s c(leaf)] = c(root),
and lo_l <= c(leaf) makes E[X] <= VR.  Markov's inequality gives
P(X >= 2^beta VR) <= 2^-beta, so over t independent trials
P(min_i 2^-beta X_i > VR) <= 2^(-beta t): the reported lower bound holds with
confidence 1 - 2^(-beta t).  Balancing the sampled violations keeps the X_i
close to each other; the guarantee does not depend on it.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the n-th output (n = 0, 1, ...) of the generator
seeded with s is mix(s + (n + 1) g mod 2^64), g = 0x9E3779B97F4A7C15, with
mix(z) = z ^ (z >> 31) after z = (z ^ (z >> 30)) 0xBF58476D1CE4E5B9 and
z = (z ^ (z >> 27)) 0x94D049BB133111EB (products mod 2^64).  A uniform double
is (output >> 11) 2^-53.  Draw n of a trial: (trial << 40) | (split << 34) |
(point << 10) | coordinate; the coin of a split uses point 2^24 - 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .counter import count
from .slr import unsafe_points

_M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
COIN_POINT = (1 << 24) - 1


def splitmix64(seed, n):
    """n-th output(s) of SplitMix64 seeded with ``seed`` (n: int or uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (np.asarray(n, dtype=np.uint64) + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def draw_index(trial, split, point, coord):
    return (np.uint64(trial) << np.uint64(40)) | (np.uint64(split) << np.uint64(34)) | \
        (np.asarray(point, dtype=np.uint64) << np.uint64(10)) | np.asarray(coord, dtype=np.uint64)


def uniform(seed, trial, split, n_points, d):
    """(n_points, d) uniform doubles in [0, 1) of one split's sample."""
    k = np.arange(n_points, dtype=np.uint64)[:, None]
    i = np.arange(d, dtype=np.uint64)[None, :]
    return (splitmix64(seed, draw_index(trial, split, k, i)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def coin(seed, trial, split):
    """0: keep the lower half, 1: the upper half."""
    return int(splitmix64(seed, draw_index(trial, split, COIN_POINT, 0)) >> np.uint64(63))


def widest_side(lo, hi):
    w = np.asarray(hi, np.float64) - np.asarray(lo, np.float64)
    return int(np.argmax(w)), float(np.max(w))


def volume_ratio(lo, hi, a, b):
    """vol(leaf) / vol(root) over the dimensions of nonzero root width, multiplied in index order."""
    r = 1.0
    for i in range(len(a)):
        wa = float(b[i]) - float(a[i])
        if wa > 0.0:
            r = r * ((float(hi[i]) - float(lo[i])) / wa)
    return r


@dataclass
class Trial:
    splits: int
    leaf_lo: np.ndarray
    leaf_hi: np.ndarray
    unsafe_lo: int
    unsafe_hi: int
    volume: float
    estimate: float
    estimate_hi: float
    samples_unsafe: int
    dims: list = field(default_factory=list)
    points: list = field(default_factory=list)     # float32 split points
    coins: list = field(default_factory=list)


@dataclass
class ApproxResult:
    vr_lower: float
    confidence: float
    vr_mean: float
    trials: list


def one_trial(net, a, b, prop, trial, splits, samples, leaf_depth, seed):
    lo = np.asarray(a, np.float32).copy()
    hi = np.asarray(b, np.float32).copy()
    d = lo.shape[0]
    s = 0
    n_uns = 0
    dims, pts, coins = [], [], []
    for j in range(splits):
        i, w = widest_side(lo, hi)
        if w <= 0.0:
            break
        u = uniform(seed, trial, j, samples, d)
        lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
        x = lo64 + (hi64 - lo64) * u                  # numpy: one rounding per operation
        bad = unsafe_points(net, prop, x)
        v = np.sort(x[bad, i])
        n_uns += int(v.shape[0])
        m64 = v[(v.shape[0] - 1) // 2] if v.shape[0] else 0.5 * (lo64[i] + hi64[i])
        m = np.float32(m64)
        if not (lo[i] < m < hi[i]):
            m = np.float32(0.5 * (lo64[i] + hi64[i]))
            if not (lo[i] < m < hi[i]):
                break
        c = coin(seed, trial, j)
        if c == 0:
            hi[i] = m
        else:
            lo[i] = m
        s += 1
        dims.append(i)
        pts.append(m)
        coins.append(c)
    r = count(net, lo, hi, prop, leaf_depth)
    vol = volume_ratio(lo, hi, a, b)
    est = float(np.ldexp(float(r.unsafe_lo) * vol, s - leaf_depth))
    est_hi = float(np.ldexp(float(r.unsafe_hi) * vol, s - leaf_depth))
    return Trial(s, lo, hi, r.unsafe_lo, r.unsafe_hi, vol, est, est_hi, n_uns, dims, pts, coins)


def count_approx(net, a, b, prop, trials=8, splits=10, samples=4096, leaf_depth=12, beta=1.0, seed=0):
    """CountingProVe_SLR: the lower bound min_i 2^-beta X_i of the violation rate,
    its confidence 1 - 2^(-beta trials) and the mean of the X_i."""
    ts = [one_trial(net, a, b, prop, k, splits, samples, leaf_depth, seed) for k in range(trials)]
    est = [t.estimate for t in ts]
    return ApproxResult(min(est) * 2.0 ** -beta, 1.0 - 2.0 ** (-beta * trials), sum(est) / len(est), ts)
