"""Symbolic Linear Relaxation bound propagation, FP64 (test infrastructure only).

Conventions
  * A network has K affine layers W_k (n_k x n_{k-1}), b_k, with ReLU after
    every layer but the last.
  * An input box is [a, b] (float64 copies of the float32 inputs).
  * A symbolic equation over the input x is a row (g_1..g_d, g_0): x -> g.x + g_0,
    stored with the constant in the LAST column.  Every hidden neuron keeps two
    such equations, an upper one U_j and a lower one L_j (Sec. 3: "for each node
    of each hidden layer we store two linear equations").
  * Property rows (C, e) describe the unsafe set; they are folded into the last
    affine layer (W' = C W_K, b' = C b_K + e) so that each row r yields a lower
    bound lo_r and an upper bound hi_r of C[r].y + e[r] over the box.

All functions accept a leading batch axis over boxes; each box is processed
independently with exactly the steps written here.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

SAFE, UNSAFE, UNDECIDED = 0, 1, 2


# ---------------------------------------------------------------------------
# Concretisation (Sec. 2.2: concrete lower/upper bound of a symbolic equation)
# ---------------------------------------------------------------------------

def concretize(E, a, b):
    """Min and max over the box [a, b] of every affine form in E.

    E: (..., n, d+1) with the constant in the last column; a, b: (..., d).
    For an affine g.x + g_0 over a box with centre m = (a+b)/2 and radius
    r = (b-a)/2, the minimum is g_0 + g.m - |g|.r and the maximum is
    g_0 + g.m + |g|.r (each coordinate independently at an endpoint).
    """
    g = E[..., :-1]
    g0 = E[..., -1]
    m = (a + b) / 2
    r = (b - a) / 2
    c = g0 + (g @ m[..., :, None])[..., 0]
    s = (np.abs(g) @ r[..., :, None])[..., 0]
    return c - s, c + s


def _pos(W):
    return np.where(W > 0, W, W * 0)


def _neg(W):
    return np.where(W < 0, W, W * 0)


def fold_property(net, prop):
    """Layers with the property rows folded into the last one (Sec. 3 check).

    Returns lists (W', b') where W'_K = C W_K and b'_K = C b_K + e, computed
    in the dtype of the inputs (float64 or exact).  Without a property the
    network's own last layer is kept (per-output bounds).
    """
    Ws = [np.asarray(w) for w in net.W]
    bs = [np.asarray(x) for x in net.b]
    if prop is not None:
        C = np.asarray(prop.C)
        e = np.asarray(prop.e)
        Ws[-1] = C @ Ws[-1]
        bs[-1] = C @ bs[-1] + e
    return Ws, bs


def _acts(net):
    """Activation of each hidden layer ('relu' unless the network says otherwise)."""
    act = list(getattr(net, "act", None) or [])
    return act if act else ["relu"] * (len(net.W) - 1)


def _as64(net, prop):
    class _N:
        pass
    n = _N()
    n.W = [np.asarray(w, dtype=np.float64) for w in net.W]
    n.b = [np.asarray(x, dtype=np.float64) for x in net.b]
    n.act = _acts(net)
    p = None
    if prop is not None:
        p = _N()
        p.C = np.asarray(prop.C, dtype=np.float64)
        p.e = np.asarray(prop.e, dtype=np.float64)
        p.strict = np.asarray(prop.strict)
        p.rows_per_clause = np.asarray(prop.rows_per_clause)
    return n, p


def to_exact(net, prop, a, b):
    """Exact-rational copies (object arrays of Fraction) of float inputs."""
    fr = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])

    class _N:
        pass
    n = _N()
    n.W = [fr(np.asarray(w, dtype=np.float64)) for w in net.W]
    n.b = [fr(np.asarray(x, dtype=np.float64)) for x in net.b]
    p = None
    if prop is not None:
        p = _N()
        p.C = fr(np.asarray(prop.C, dtype=np.float64))
        p.e = fr(np.asarray(prop.e, dtype=np.float64))
        p.strict = np.asarray(prop.strict)
        p.rows_per_clause = np.asarray(prop.rows_per_clause)
    return n, p, fr(np.asarray(a, dtype=np.float64)), fr(np.asarray(b, dtype=np.float64))


# ---------------------------------------------------------------------------
# Naive interval propagation (Moore intervals; Sec. 2.2 and the Exact Count
# baseline of Sec. 4)
# ---------------------------------------------------------------------------

def interval_forward(net, a, b, prop=None, exact=False):
    """Moore interval bounds.

    Returns (lo, hi, pre) where lo, hi bound the property rows (or the outputs
    without a property) and pre[k] = (l, u) are the pre-activation bounds of
    hidden layer k+1.
    """
    acts = _acts(net)
    if not exact:
        net, prop = _as64(net, prop)
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
    Ws, bs = fold_property(net, prop)
    l, u = a, b
    pre = []
    for k, (W, bb) in enumerate(zip(Ws, bs)):
        Wp, Wn = _pos(W), _neg(W)
        l2 = (Wp @ l[..., :, None])[..., 0] + (Wn @ u[..., :, None])[..., 0] + bb
        u2 = (Wp @ u[..., :, None])[..., 0] + (Wn @ l[..., :, None])[..., 0] + bb
        if k < len(Ws) - 1:
            pre.append((l2, u2))
            if acts[k] == "relu":
                l, u = np.where(l2 > 0, l2, l2 * 0), np.where(u2 > 0, u2, u2 * 0)
            else:                                  # monotone: the image of [l2, u2]
                l, u = act_value(acts[k], l2), act_value(acts[k], u2)
        else:
            l, u = l2, u2
    return l, u, pre


# ---------------------------------------------------------------------------
# Symbolic Linear Relaxation (Sec. 2.2, Eq. 1, as used in Sec. 3)
# ---------------------------------------------------------------------------

def _relax(U, L, ll, ul, lu, uu, alpha, mode):
    """Relax one hidden layer's ReLUs; returns the post-activation (U, L).

    ll, ul: min and max of the lower equation L_j over the box;
    lu, uu: min and max of the upper equation U_j over the box.

    mode 'neurify' (default reading of Eq. 1): each equation is relaxed with
    its own concrete bounds.
      stable active   (ll >= 0): U_j, L_j unchanged
      stable inactive (uu <= 0): U_j = L_j = 0
      unstable, upper: U_j unchanged if lu >= 0, else the chord
                       s (U_j - lu), s = uu / (uu - lu)
      unstable, lower: 0 if ul <= 0, else alpha_j L_j with
                       alpha_j = ul / (ul - ll) unless supplied (any value in
                       [0, 1] is sound since relu(z) >= alpha z >= alpha L_j)
    mode 'paper_literal': one pair (l, u) = (ll, uu) for both equations, so
      the unstable case is U_j = s (U_j - l), L_j = s L_j, s = u / (u - l).
    """
    zero = U * 0
    if mode == "paper_literal":
        lo_, up_ = ll, uu
        active = lo_ >= 0
        inactive = (~active) & (up_ <= 0)
        unstable = ~(active | inactive)
        den = np.where(unstable, up_ - lo_, up_ * 0 + 1)
        s = np.where(unstable, up_ / den, up_ * 0)
        Uc = U * s[..., None]
        Uc[..., -1] = Uc[..., -1] - s * lo_
        Lc = L * s[..., None]
        U2 = np.where(active[..., None], U, np.where(unstable[..., None], Uc, zero))
        L2 = np.where(active[..., None], L, np.where(unstable[..., None], Lc, zero))
        return U2, L2

    active = ll >= 0
    inactive = (~active) & (uu <= 0)
    unstable = ~(active | inactive)
    # upper equation
    chord = unstable & (lu < 0)
    den_u = np.where(chord, uu - lu, uu * 0 + 1)
    s = np.where(chord, uu / den_u, uu * 0)
    Uc = U * s[..., None]
    Uc[..., -1] = Uc[..., -1] - s * lu
    U_unst = np.where(chord[..., None], Uc, U)
    # lower equation
    lin = unstable & (ul > 0)
    if alpha is None:
        den_l = np.where(lin, ul - ll, ul * 0 + 1)
        al = np.where(lin, ul / den_l, ul * 0)
    else:
        al = np.where(lin, alpha, ul * 0)
    L_unst = np.where(lin[..., None], L * al[..., None], zero)
    U2 = np.where(active[..., None], U, np.where(unstable[..., None], U_unst, zero))
    L2 = np.where(active[..., None], L, np.where(unstable[..., None], L_unst, zero))
    return U2, L2


# ---------------------------------------------------------------------------
# S-shaped activations (tanh, logistic sigmoid): Sec. 3 names activations
# other than ReLU only as an extension; the relaxation below is this build's
# restatement for monotone functions that are convex below 0 and concave
# above it, with a derivative largest at 0 and falling off on both sides.
# ---------------------------------------------------------------------------

def act_value(name, z):
    if name == "tanh":
        return np.tanh(z)
    if name == "sigmoid":
        return 1.0 / (1.0 + np.exp(-z))
    return np.maximum(z, 0.0)


def act_slope(name, z):
    if name == "tanh":
        t = np.tanh(z)
        return 1.0 - t * t
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 - s)


def _relax_s(U, L, ll, uu, name):
    """Relax one hidden layer of an S-shaped activation s over z in [l, u] = [ll, uu].

      l >= 0 (s concave): upper = tangent at m = (l + u) / 2, lower = chord;
      u <= 0 (s convex):  upper = chord, lower = tangent at m;
      l < 0 < u:          both with slope lam = min(s'(l), s'(u)), the upper
                          through (u, s(u)), the lower through (l, s(l));
      l == u:             both the constant s(l).
    A tangent lies below a convex function and above a concave one, a chord
    the other way round; in the straddling case s' >= lam on [l, u] (s' is
    largest at 0 and falls off on both sides), so the upper line minus s
    decreases to 0 at u and the lower line minus s increases from 0 at l.
    The new equations are U' = a_u U + b_u and L' = a_l L + b_l (a >= 0, and
    l <= L, U <= u on the box).
    """
    l, u = ll, uu
    sl, su = act_value(name, l), act_value(name, u)
    width = u - l
    pos = width > 0
    chord = np.where(pos, (su - sl) / np.where(pos, width, 1.0), 0.0)
    m = 0.5 * (l + u)
    tm = act_slope(name, m)
    lam = np.minimum(act_slope(name, l), act_slope(name, u))
    concave = l >= 0
    convex = (~concave) & (u <= 0)
    # upper line a_u z + b_u
    a_u = np.where(concave, tm, np.where(convex, chord, lam))
    b_u = np.where(concave, act_value(name, m) - tm * m, np.where(convex, sl - chord * l, su - lam * u))
    # lower line a_l z + b_l
    a_l = np.where(concave, chord, np.where(convex, tm, lam))
    b_l = np.where(concave, sl - chord * l, np.where(convex, act_value(name, m) - tm * m, sl - lam * l))
    a_u = np.where(pos, a_u, 0.0)
    a_l = np.where(pos, a_l, 0.0)
    b_u = np.where(pos, b_u, sl)
    b_l = np.where(pos, b_l, sl)
    U2 = U * a_u[..., None]
    U2[..., -1] = U2[..., -1] + b_u
    L2 = L * a_l[..., None]
    L2[..., -1] = L2[..., -1] + b_l
    return U2, L2


def slr_forward(net, a, b, prop=None, alpha=None, mode="neurify", exact=False):
    """SLR bounds of the property rows (or outputs) over each box.

    a, b: (B, d) or (d,).  alpha: optional list, one (B, n_k) array of lower
    slopes per hidden layer.  Returns (lo, hi, pre) where pre[k] =
    (ll, ul, lu, uu) are the concrete bounds of hidden layer k+1's
    pre-activation equations.

    Steps (Sec. 3): layer 1 gives U = L = [W_1 | b_1]; then for each hidden
    layer: concretise both equations over the box, relax the ReLU (Eq. 1),
    and push both equations through the next affine layer with
    U' = W+ U + W- L + b, L' = W+ L + W- U + b (W+ = max(W,0), W- = min(W,0)).
    The row bounds are lo = min L', hi = max U' over the box.
    """
    acts = _acts(net)
    if any(x != "relu" for x in acts) and (exact or alpha is not None):
        raise ValueError("S-shaped activations: no exact rationals and no supplied slopes")
    if not exact:
        net, prop = _as64(net, prop)
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
    squeeze = a.ndim == 1
    if squeeze:
        a, b = a[None], b[None]
    Ws, bs = fold_property(net, prop)
    nb = a.shape[0]
    E1 = np.concatenate([Ws[0], bs[0][:, None]], axis=1)
    U = np.broadcast_to(E1, (nb,) + E1.shape).copy()
    L = U.copy()
    pre = []
    for k in range(1, len(Ws)):
        ll, ul = concretize(L, a, b)
        lu, uu = concretize(U, a, b)
        pre.append((ll, ul, lu, uu))
        name = acts[k - 1]
        if name == "relu":
            U, L = _relax(U, L, ll, ul, lu, uu, None if alpha is None else alpha[k - 1], mode)
        else:
            U, L = _relax_s(U, L, ll, uu, name)
        W, bb = Ws[k], bs[k]
        Wp, Wn = _pos(W), _neg(W)
        U2 = Wp @ U + Wn @ L
        L2 = Wp @ L + Wn @ U
        U2[..., -1] = U2[..., -1] + bb
        L2[..., -1] = L2[..., -1] + bb
        U, L = U2, L2
    lo = concretize(L, a, b)[0]
    hi = concretize(U, a, b)[1]
    if squeeze:
        lo, hi = lo[0], hi[0]
        pre = [tuple(x[0] for x in p) for p in pre]
    return lo, hi, pre


# ---------------------------------------------------------------------------
# Classification (Sec. 3: R subset of Y -> unsafe, R disjoint from Y -> safe)
# ---------------------------------------------------------------------------

def classify(lo, hi, prop):
    """Classify boxes from their row bounds.

    The unsafe set Y is an OR over clauses of an AND over rows
    (C[r].y + e[r] >= 0, or > 0 where strict).  A box is UNSAFE when some
    clause has every row provably satisfied on it (lo_r >= 0, > 0 if strict),
    i.e. R is inside Y; SAFE when every clause has a row provably violated
    (hi_r < 0, <= 0 if strict), i.e. R does not meet Y; otherwise UNDECIDED.
    """
    strict = np.asarray(prop.strict).astype(bool)
    row_in = np.where(strict, lo > 0, lo >= 0)
    row_out = np.where(strict, hi <= 0, hi < 0)
    nb = row_in.shape[:-1]
    any_clause_in = np.zeros(nb, dtype=bool)
    all_clause_out = np.ones(nb, dtype=bool)
    r0 = 0
    for nr in np.asarray(prop.rows_per_clause):
        nr = int(nr)
        any_clause_in |= np.all(row_in[..., r0:r0 + nr], axis=-1)
        all_clause_out &= np.any(row_out[..., r0:r0 + nr], axis=-1)
        r0 += nr
    cls = np.full(nb, UNDECIDED, dtype=np.int8)
    cls[all_clause_out] = SAFE
    cls[any_clause_in] = UNSAFE
    return cls


# ---------------------------------------------------------------------------
# Concrete evaluation (for sampling checks in the tests)
# ---------------------------------------------------------------------------

def forward_points(net, x, prop=None):
    """FP64 forward pass of points x (N, d); returns (rows or outputs, hidden pre-activations)."""
    h = np.asarray(x, dtype=np.float64)
    pre = []
    K = len(net.W)
    acts = _acts(net)
    for k in range(K):
        z = h @ np.asarray(net.W[k], dtype=np.float64).T + np.asarray(net.b[k], dtype=np.float64)
        if k < K - 1:
            pre.append(z)
            h = act_value(acts[k], z)
        else:
            h = z
    if prop is not None:
        h = h @ np.asarray(prop.C, dtype=np.float64).T + np.asarray(prop.e, dtype=np.float64)
    return h, pre


def unsafe_points(net, prop, x):
    """Boolean mask: which points x lie in the unsafe set (FP64 forward pass)."""
    rows, _ = forward_points(net, x, prop)
    strict = np.asarray(prop.strict).astype(bool)
    sat = np.where(strict, rows > 0, rows >= 0)
    out = np.zeros(rows.shape[0], dtype=bool)
    r0 = 0
    for nr in np.asarray(prop.rows_per_clause):
        out |= np.all(sat[:, r0:r0 + int(nr)], axis=1)
        r0 += int(nr)
    return out
