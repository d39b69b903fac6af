"""Central finite differences of the SLR row bounds (test infrastructure only).

The objective is J = sum_r (w_hi[r] hi_r + w_lo[r] lo_r) over one box's SLR row
bounds (Sec. 2.2, Eq. 1; Sec. 3).  Derivatives are taken by central
differences in float64 with step h on the lower ReLU slopes alpha (any value
in [0, 1] keeps the relaxation sound), the box endpoints, the weights and the
biases.  A coordinate is reported as a kink (NaN) when the estimates with
steps h and h/2 disagree, i.e. a ReLU case or a sign of a coefficient changes
inside the stencil; the adjoint is compared only away from kinks.
"""
from __future__ import annotations

import numpy as np

from .slr import slr_forward


def objective(net, lo, hi, prop, alpha, w_hi, w_lo):
    """J for one box (lo, hi: (d,)), alpha: list of (n_k,) arrays or None."""
    a = None if alpha is None else [np.asarray(x, dtype=np.float64)[None] for x in alpha]
    rlo, rhi, _ = slr_forward(net, np.asarray(lo, np.float64)[None], np.asarray(hi, np.float64)[None], prop, alpha=a)
    return float(np.dot(w_hi, rhi[0]) + np.dot(w_lo, rlo[0]))


def _central(f, x0, h):
    g = np.empty_like(x0)
    for i in range(x0.size):
        e = np.zeros_like(x0)
        e.flat[i] = h
        g.flat[i] = (f(x0 + e) - f(x0 - e)) / (2 * h)
    return g


def fd_gradients(net, lo, hi, prop, alpha, w_hi, w_lo, h=1e-3, tol=1e-6, w_idx=None, alpha_idx=None,
                 box_idx=None):
    """Central-difference gradients of J; entries at kinks are NaN.

    alpha: list of per-layer slope arrays, or None for the slopes u/(u-l)
    (then J is differentiated through that formula and 'alpha' is empty).
    w_idx: optional dict layer -> flat indices of the weights to difference
    (the others are NaN); all weights when None.
    alpha_idx, box_idx: optional indices (into the concatenated slopes, and
    into the input dimensions for both box endpoints) to difference; the
    others are NaN; all when None.
    Returns dict with 'alpha' (list per hidden layer), 'lo', 'hi', 'W', 'b'.
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    free = alpha is not None
    alpha = [np.asarray(a, np.float64) for a in alpha] if free else None
    sizes = [a.size for a in alpha] if free else []

    def split(v):
        out, o = [], 0
        for s in sizes:
            out.append(v[o:o + s])
            o += s
        return out

    def both(f, x0, idx=None):
        if idx is None:
            g1 = _central(f, x0, h)
            g2 = _central(f, x0, h / 2)
        else:
            g1 = np.full_like(x0, np.nan)
            g2 = np.full_like(x0, np.nan)
            for i in idx:
                e = np.zeros_like(x0)
                e.flat[i] = 1.0
                g1.flat[i] = (f(x0 + h * e) - f(x0 - h * e)) / (2 * h)
                g2.flat[i] = (f(x0 + h / 2 * e) - f(x0 - h / 2 * e)) / h
        scale = 1.0 + np.abs(g1)
        return np.where(np.abs(g1 - g2) <= tol * scale + 1e-9, g1, np.nan)

    out = {}
    if free:
        a0 = np.concatenate(alpha) if alpha else np.zeros(0)
        out["alpha"] = split(both(lambda v: objective(net, lo, hi, prop, split(v), w_hi, w_lo), a0, alpha_idx))
    else:
        out["alpha"] = []
    out["lo"] = both(lambda v: objective(net, v, hi, prop, alpha, w_hi, w_lo), lo, box_idx)
    out["hi"] = both(lambda v: objective(net, lo, v, prop, alpha, w_hi, w_lo), hi, box_idx)

    class _N:
        pass
    Ws, bs = [], []
    for k in range(len(net.W)):
        W0 = np.asarray(net.W[k], np.float64)
        b0 = np.asarray(net.b[k], np.float64)

        def fw(v, k=k, W0=W0):
            n = _N()
            n.W = [np.asarray(x, np.float64) for x in net.W]
            n.b = [np.asarray(x, np.float64) for x in net.b]
            n.W[k] = v.reshape(W0.shape)
            return objective(n, lo, hi, prop, alpha, w_hi, w_lo)

        def fb(v, k=k):
            n = _N()
            n.W = [np.asarray(x, np.float64) for x in net.W]
            n.b = [np.asarray(x, np.float64) for x in net.b]
            n.b[k] = v
            return objective(n, lo, hi, prop, alpha, w_hi, w_lo)

        idx = None if w_idx is None else w_idx.get(k, [])
        Ws.append(both(fw, W0.ravel(), idx).reshape(W0.shape))
        bs.append(both(fb, b0, None if w_idx is None else list(range(b0.size)) if k in w_idx else []))
    out["W"] = Ws
    out["b"] = bs
    return out


def default_alpha(net, lo, hi, prop=None):
    """The default lower slopes u_l / (u_l - l_l) of each unstable neuron (0 elsewhere)."""
    _, _, pre = slr_forward(net, np.asarray(lo, np.float64), np.asarray(hi, np.float64), prop)
    out = []
    for ll, ul, lu, uu in pre:
        unst = (ll < 0) & (uu > 0) & (ul > 0)
        out.append(np.where(unst, ul / np.where(unst, ul - ll, 1.0), 0.0))
    return out
