"""Exact count by bisection, level by level, FP64 (test infrastructure only).

Alg. 1 ("Exact Count") keeps a set of unknown boxes, classifies each one and
either adds its volume (unsafe), drops it (safe) or bisects it (undecided).
Sec. 3 evaluates all boxes of one level of the branch-and-bound tree
together.  This module does exactly that, breadth-first, with a depth cap D:

  * a box at depth t is named by a path code, the t bits of the halves chosen
    at splits 0..t-1 (first split in the most significant bit);
  * the split dimension of split j is the same for every box of a level (the
    widest side, ties to the lowest index, Sec. 2.2 "evenly dividing the
    interval into two consecutive sub-intervals"), so one schedule serves all;
  * an UNSAFE box at depth t adds 2^(D-t) units (one unit = 2^-D of the root
    volume); an UNDECIDED box at depth D adds one unit to the undecided
    count; the violation rate then lies in [lo, lo + und] / 2^D.

With a ``split`` callable the dimension is chosen per box instead (e.g. the
gradient rule of ``split.py``); each box then carries its own half indices
k_i and split counts c_i, and spans [a_i + w_i k_i 2^-c_i, a_i + w_i (k_i+1) 2^-c_i]
as before.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .slr import SAFE, UNSAFE, UNDECIDED, classify, slr_forward, interval_forward


def split_schedule(a, b, D):
    """Dimension split at each of the D levels ("widest first", ties to lowest index).

    Widths w_i = b_i - a_i are taken in float64 from the float32 root box; after
    c_i splits dimension i has width w_i 2^-c_i.
    """
    w = np.asarray(b, dtype=np.float64) - np.asarray(a, dtype=np.float64)
    c = np.zeros(w.shape[0], dtype=np.int64)
    sched = []
    for _ in range(D):
        score = w * np.ldexp(1.0, -c)
        i = int(np.argmax(score))          # first maximum: lowest index on ties
        sched.append(i)
        c[i] += 1
    return np.array(sched, dtype=np.int64)


def decode(codes, t, sched, a, b):
    """Float64 endpoints of the boxes with the given depth-t path codes.

    Bit (t-1-j) of a code is the half (0 lower, 1 upper) taken at split j along
    dimension sched[j].  Dimension i, split c_i times into halves with index k_i,
    spans [a_i + w_i k_i 2^-c_i, a_i + w_i (k_i+1) 2^-c_i].
    """
    codes = np.asarray(codes, dtype=np.int64)
    a64 = np.asarray(a, dtype=np.float64)
    b64 = np.asarray(b, dtype=np.float64)
    d = a64.shape[0]
    n = codes.shape[0]
    k = np.zeros((n, d), dtype=np.int64)
    c = np.zeros(d, dtype=np.int64)
    for j in range(t):
        bit = (codes >> (t - 1 - j)) & 1
        i = int(sched[j])
        k[:, i] = 2 * k[:, i] + bit
        c[i] += 1
    w = b64 - a64
    scale = np.ldexp(1.0, -c)
    lo = a64 + w * (k * scale)
    hi = a64 + w * ((k + 1) * scale)
    return lo, hi


@dataclass
class CountResult:
    unsafe_lo: int
    unsafe_hi: int
    depth: int
    levels: list = field(default_factory=list)      # per level: dict(boxes, safe, unsafe, undecided)
    leaves: list = field(default_factory=list)      # (code, depth, class) when collected
    leaf_boxes: list = field(default_factory=list)  # per-box splits: (lo, hi) of each collected leaf

    @property
    def boxes(self):
        return sum(lv["boxes"] for lv in self.levels)


def count(net, a, b, prop, D, mode="neurify", bound="slr", collect_leaves=False,
          batch=8192, max_boxes=None, split=None):
    """Exact-count bracket [unsafe_lo, unsafe_hi] in units of 2^-D of the root box.

    bound='slr' uses symbolic linear relaxation; bound='interval' uses naive
    Moore intervals (the paper's Exact Count baseline).  ``max_boxes`` stops
    after that many box evaluations (a bounded sample used only for timing)
    and returns the partial result.  ``split``: None splits the widest side
    (one schedule for every box of a level); a callable
    split(t, paths, lo, hi) -> dims gives the dimension of each UNDECIDED box
    of level t (paths: their path codes; lo, hi: float64 endpoints).
    """
    if split is not None:
        return _count_per_box(net, a, b, prop, D, mode, bound, collect_leaves, batch, split)
    sched = split_schedule(a, b, D)
    frontier = np.zeros(1, dtype=np.int64)
    lo = 0
    und = 0
    res = CountResult(0, 0, D)
    evaluated = 0
    for t in range(D + 1):
        nxt = []
        lv = dict(boxes=int(frontier.shape[0]), safe=0, unsafe=0, undecided=0)
        for s in range(0, frontier.shape[0], batch):
            codes = frontier[s:s + batch]
            blo, bhi = decode(codes, t, sched, a, b)
            if bound == "slr":
                rlo, rhi, _ = slr_forward(net, blo, bhi, prop, mode=mode)
            else:
                rlo, rhi, _ = interval_forward(net, blo, bhi, prop)
            cls = classify(rlo, rhi, prop)
            n_uns = int(np.count_nonzero(cls == UNSAFE))
            lv["unsafe"] += n_uns
            lv["safe"] += int(np.count_nonzero(cls == SAFE))
            und_codes = codes[cls == UNDECIDED]
            lv["undecided"] += int(und_codes.shape[0])
            lo += n_uns << (D - t)
            if t < D:
                nxt.append(2 * und_codes)
                nxt.append(2 * und_codes + 1)
            else:
                und += int(und_codes.shape[0])
            if collect_leaves:
                for cd, cl in zip(codes.tolist(), cls.tolist()):
                    if cl != UNDECIDED or t == D:
                        res.leaves.append((cd, t, cl))
            evaluated += codes.shape[0]
            if max_boxes is not None and evaluated >= max_boxes:
                res.levels.append(lv)
                res.unsafe_lo, res.unsafe_hi = lo, lo + und
                return res
        res.levels.append(lv)
        if t < D:
            frontier = np.concatenate(nxt) if nxt else np.zeros(0, dtype=np.int64)
            if frontier.shape[0] == 0:
                for _ in range(t + 1, D + 1):
                    res.levels.append(dict(boxes=0, safe=0, unsafe=0, undecided=0))
                break
    res.unsafe_lo, res.unsafe_hi = lo, lo + und
    return res


def _count_per_box(net, a, b, prop, D, mode, bound, collect_leaves, batch, split):
    """``count`` with a split dimension chosen per box."""
    a64 = np.asarray(a, dtype=np.float64)
    w = np.asarray(b, dtype=np.float64) - a64
    d = a64.shape[0]
    paths = np.zeros(1, dtype=np.int64)
    K = np.zeros((1, d), dtype=np.int64)      # half index along each dimension
    C = np.zeros((1, d), dtype=np.int64)      # splits along each dimension
    lo = 0
    und = 0
    res = CountResult(0, 0, D)
    for t in range(D + 1):
        nxt = []
        lv = dict(boxes=int(paths.shape[0]), safe=0, unsafe=0, undecided=0)
        for s in range(0, paths.shape[0], batch):
            p, k, c = paths[s:s + batch], K[s:s + batch], C[s:s + batch]
            scale = np.ldexp(1.0, -c)
            blo = a64 + w * (k * scale)
            bhi = a64 + w * ((k + 1) * scale)
            if bound == "slr":
                rlo, rhi, _ = slr_forward(net, blo, bhi, prop, mode=mode)
            else:
                rlo, rhi, _ = interval_forward(net, blo, bhi, prop)
            cls = classify(rlo, rhi, prop)
            n_uns = int(np.count_nonzero(cls == UNSAFE))
            lv["unsafe"] += n_uns
            lv["safe"] += int(np.count_nonzero(cls == SAFE))
            u = cls == UNDECIDED
            lv["undecided"] += int(np.count_nonzero(u))
            lo += n_uns << (D - t)
            if t < D:
                if np.any(u):
                    dims = np.asarray(split(t, p[u], blo[u], bhi[u]), dtype=np.int64)
                    rows = np.arange(dims.shape[0])
                    k0 = k[u].copy()
                    c1 = c[u].copy()
                    k0[rows, dims] *= 2
                    c1[rows, dims] += 1
                    k1 = k0.copy()
                    k1[rows, dims] += 1
                    nxt.append((2 * p[u], k0, c1))
                    nxt.append((2 * p[u] + 1, k1, c1))
            else:
                und += int(np.count_nonzero(u))
            if collect_leaves:
                for j, (cd, cl) in enumerate(zip(p.tolist(), cls.tolist())):
                    if cl != UNDECIDED or t == D:
                        res.leaves.append((cd, t, cl))
                        res.leaf_boxes.append((blo[j], bhi[j]))
        res.levels.append(lv)
        if t < D:
            if not nxt:
                for _ in range(t + 1, D + 1):
                    res.levels.append(dict(boxes=0, safe=0, unsafe=0, undecided=0))
                break
            paths = np.concatenate([x[0] for x in nxt])
            K = np.concatenate([x[1] for x in nxt])
            C = np.concatenate([x[2] for x in nxt])
    res.unsafe_lo, res.unsafe_hi = lo, lo + und
    return res
