"""The gradient split rule: a split dimension per box (test infrastructure only).

Sec. 2.2 bisects an undecided box into two halves of one input interval and
leaves open which interval.  Besides the widest side (``counter.split_schedule``)
the counter offers a data-dependent rule, read as follows.

Decision loss M of one box, from its row bounds (lo_r, hi_r) and the clauses
of the unsafe set (Sec. 3: OR over clauses of AND over rows):

  safe gap    s = sum over clauses c of max(min_{r in c} hi_r, 0)
  unsafe gap  u = min over clauses c of max(-min_{r in c} lo_r, 0)   (c*: the first argmin)
  M = s  if s <= u  (pushing the box towards SAFE: every clause needs a row with hi < 0)
  M = max(-min_{r in c*} lo_r, 0) otherwise  (towards UNSAFE: every row of c* with lo >= 0)

M is piecewise linear in the row bounds; its derivative is taken with the
selections (direction, clause, the first row attaining each minimum) fixed at
the box, i.e. as the linear functional J = sum w_hi hi + w_lo lo of
``grad.objective``.

  * dM/dr_i: derivative along the box radius, lo_i = m_i - r_i and
    hi_i = m_i + r_i, by central differences at the slopes u/(u-l), with a
    step h r_i relative to the radius (an absolute step could exceed the
    radius of a deep box and turn it inside out);
  * split set S: the (at most 16) dimensions with the largest |dM/dr_i| w_i at
    the root box (w the root widths; ties to the lowest index), ascending;
  * each UNDECIDED box splits the dimension i of S with the largest
    |dM/dr_i| r_i for its own radius (the first in S on ties).

The first-order change of M when dimension i is halved is about
(dM/dr_i) r_i / 2, so the rule halves the side that is predicted to move the
box most towards a decision.
"""
from __future__ import annotations

import numpy as np

from .grad import objective
from .slr import slr_forward


def decision_weights(rlo, rhi, prop):
    """(w_hi, w_lo, M) of one box's row bounds (rlo, rhi: (R,))."""
    R = rlo.shape[0]
    w_hi = np.zeros(R)
    w_lo = np.zeros(R)
    ends = np.cumsum(np.asarray(prop.rows_per_clause, dtype=np.int64))
    starts = ends - np.asarray(prop.rows_per_clause, dtype=np.int64)
    safe_gap = 0.0
    unsafe_gap = np.inf
    best = -1
    for c, (r0, r1) in enumerate(zip(starts, ends)):
        safe_gap += max(float(np.min(rhi[r0:r1])), 0.0)
        ug = max(-float(np.min(rlo[r0:r1])), 0.0)
        if ug < unsafe_gap:
            unsafe_gap = ug
            best = c
    if safe_gap <= unsafe_gap:
        for r0, r1 in zip(starts, ends):
            rh = r0 + int(np.argmin(rhi[r0:r1]))       # first minimum
            if rhi[rh] > 0:
                w_hi[rh] += 1.0
        return w_hi, w_lo, safe_gap
    r0, r1 = starts[best], ends[best]
    rl = r0 + int(np.argmin(rlo[r0:r1]))
    if rlo[rl] < 0:
        w_lo[rl] = -1.0
    return w_hi, w_lo, unsafe_gap


def radius_gradient(net, lo, hi, prop, dims=None, h=1e-3, tol=1e-6):
    """dM/dr_i of one box for i in dims (all when None), NaN at kinks.

    Central differences with steps h r_i and h r_i / 2 on the radius; a
    coordinate whose two estimates disagree (a ReLU case or a coefficient sign
    changes inside the stencil) is a kink.
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    rlo, rhi, _ = slr_forward(net, lo[None], hi[None], prop)
    w_hi, w_lo, _ = decision_weights(rlo[0], rhi[0], prop)
    dims = range(lo.size) if dims is None else dims
    g = np.full(lo.size, np.nan)
    for i in dims:
        e = np.zeros(lo.size)
        e[i] = 1.0
        s0 = h * 0.5 * (hi[i] - lo[i])
        if s0 <= 0:
            continue

        def f(s):
            return objective(net, lo - s * e, hi + s * e, prop, None, w_hi, w_lo)
        g1 = (f(s0) - f(-s0)) / (2 * s0)
        g2 = (f(s0 / 2) - f(-s0 / 2)) / s0
        if abs(g1 - g2) <= tol * (1.0 + abs(g1)) + 1e-9:
            g[i] = g1
    return g


def split_set(net, lo, hi, prop, k=16, h=1e-3):
    """S at the root box: the k dimensions of largest |dM/dr_i| w_i, ascending.

    Kinks (NaN) score as their h-step estimate: the set is a heuristic choice,
    and the comparison with the GPU's set is made on clear margins only.
    """
    scores = root_scores(net, lo, hi, prop, h)
    order = sorted(range(scores.size), key=lambda i: (-scores[i], i))
    return np.array(sorted(order[:min(k, scores.size)]), dtype=np.int64)


def root_scores(net, lo, hi, prop, h=1e-3, chunk=64):
    """|dM/dr_i| w_i at the root (central differences with step h r_i, no kink test).

    The 2d stencil boxes are bounded together, ``chunk`` at a time (the same
    per-box arithmetic as one box at a time).
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d = lo.size
    rlo, rhi, _ = slr_forward(net, lo[None], hi[None], prop)
    w_hi, w_lo, _ = decision_weights(rlo[0], rhi[0], prop)
    step = h * 0.5 * (hi - lo)
    E = np.diag(step)
    blo = np.concatenate([lo - E, lo + E])      # radius + step, then radius - step
    bhi = np.concatenate([hi + E, hi - E])
    J = np.empty(2 * d)
    for s in range(0, 2 * d, chunk):
        a, b, _ = slr_forward(net, blo[s:s + chunk], bhi[s:s + chunk], prop)
        J[s:s + chunk] = b @ w_hi + a @ w_lo
    g = np.divide(J[:d] - J[d:], 2 * step, out=np.zeros(d), where=step > 0)
    return np.abs(g) * (hi - lo)


def box_scores(net, lo, hi, prop, S, h=1e-3):
    """|dM/dr_i| r_i for i in S (kinks NaN)."""
    g = radius_gradient(net, lo, hi, prop, dims=S, h=h)
    r = 0.5 * (np.asarray(hi, np.float64) - np.asarray(lo, np.float64))
    return np.abs(g[S]) * r[S]


def gradient_split(net, prop, S, h=1e-3):
    """A ``split`` callable for ``counter.count``: per UNDECIDED box the
    dimension of S with the largest |dM/dr_i| r_i (first on ties; a kink
    scores as its central-difference estimate, step h r_i)."""
    S = np.asarray(S, dtype=np.int64)

    def choose(t, paths, lo, hi):
        out = np.empty(paths.shape[0], dtype=np.int64)
        for b in range(paths.shape[0]):
            rlo, rhi, _ = slr_forward(net, lo[b][None], hi[b][None], prop)
            w_hi, w_lo, _ = decision_weights(rlo[0], rhi[0], prop)
            best, sel = -1.0, 0
            for j, i in enumerate(S):
                r = 0.5 * (hi[b][i] - lo[b][i])
                e = np.zeros(lo.shape[1])
                e[i] = h * r
                g = (objective(net, lo[b] - e, hi[b] + e, prop, None, w_hi, w_lo)
                     - objective(net, lo[b] + e, hi[b] - e, prop, None, w_hi, w_lo)) / (2 * h * r)
                sc = abs(g) * r
                if sc > best:
                    best, sel = sc, j
            out[b] = S[sel]
        return out
    return choose
