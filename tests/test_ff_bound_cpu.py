"""The float-float product bound of the re-check's first stage, checked on the CPU.

The stage sums w_i x_i (w_i float32, x_i float64 split into float32 hi + lo)
with exact products (TwoProduct), TwoSum on the hi parts and the error terms
plus w_i lo_i summed in float32, optionally in 2 or 4 parts on neighbouring
lanes whose pairs are then added by TwoSum; the result hi + lo rounded to
float64 is claimed within gam_ff(n) sum_i |w_i| |x_i| of the exact sum (plus
an underflow term that these inputs do not reach).  Here the same float32
steps are emulated exactly (each float32 operation rounded once from its
exact rational value) and the claim is checked on random and on heavily
cancelling dot products."""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def f32(v):
    """Round an exact rational to the nearest float32 (ties to even)."""
    return F32(float(v)) if abs(Fraction(float(v)) - v) == 0 else _round32(v)


def _round32(v):
    # nearest float64 first can double-round; correct it against the two float32 neighbours
    a = F32(float(v))
    lo = np.nextafter(a, F32(-np.inf))
    hi = np.nextafter(a, F32(np.inf))
    best = min((a, lo, hi), key=lambda c: (abs(Fraction(float(c)) - v), int(np.frombuffer(c.tobytes(), np.uint32)[0]) & 1))
    return F32(best)


def fr(x):
    return Fraction(float(x))


def add(a, b):
    return f32(fr(a) + fr(b))


def sub(a, b):
    return f32(fr(a) - fr(b))


def mul(a, b):
    return f32(fr(a) * fr(b))


def fma(a, b, c):
    return f32(fr(a) * fr(b) + fr(c))


def two_sum(a, b):
    s = add(a, b)
    z = sub(s, a)
    e = add(sub(a, sub(s, z)), sub(b, z))
    return s, e


def ff_mac(w, h, l, s, e):
    p = mul(w, h)
    pe = fma(w, h, -p)
    t, se = two_sum(s, p)
    return t, fma(w, l, add(e, add(pe, se)))


def split(x):
    h = F32(x)
    lo = F32(float(x) - float(h))   # x - h is exact in float64
    return h, lo


def ff_dot(w, x, parts):
    n = len(w)
    sums = []
    for k in range(parts):
        s, e = F32(0), F32(0)
        for i in range(k * n // parts, (k + 1) * n // parts):
            h, lo = split(x[i])
            s, e = ff_mac(w[i], h, lo, s, e)
        sums.append((s, e))
    # lane pairs combined as the kernel does: by TwoSum, with the error terms in float
    while len(sums) > 1:
        nxt = []
        for (s0, e0), (s1, e1) in zip(sums[0::2], sums[1::2]):
            t, se = two_sum(s0, s1)
            nxt.append((t, add(e0, add(e1, se))))
        sums = nxt
    s, e = sums[0]
    return float(s) + float(e)       # hi + lo rounded to float64


def gam_ff(n):
    g = (n + 4) * 2.0 ** -24
    gn = (n + 2) * 2.0 ** -24
    return 4 * g * g * (1 + gn) + 2.0 ** -47


def _check(w, x, parts):
    got = Fraction(ff_dot(w, x, parts))
    exact = sum(fr(wi) * fr(xi) for wi, xi in zip(w, x))
    mag = sum(abs(fr(wi)) * abs(fr(xi)) for wi, xi in zip(w, x))
    assert abs(got - exact) <= Fraction(gam_ff(len(w))) * mag, (float(abs(got - exact) / mag), gam_ff(len(w)))
    return float(abs(got - exact) / mag)


@pytest.mark.parametrize("parts", [1, 2, 4])
def test_random_dot_products_within_the_bound(parts):
    rng = np.random.default_rng(7 + parts)
    for n in (8, 24, 50):
        for _ in range(4):
            w = rng.standard_normal(n).astype(np.float32)
            x = rng.standard_normal(n) * np.exp(rng.uniform(-6, 6, n))
            _check(w, x, parts)


@pytest.mark.parametrize("parts", [1, 4])
def test_cancelling_dot_products_within_the_bound(parts):
    """Sums whose exact value is tiny next to sum |w x|: the regime of a bound
    near zero, where the stage must not claim more accuracy than it has."""
    rng = np.random.default_rng(11)
    n = 50
    for _ in range(4):
        w = rng.standard_normal(n).astype(np.float32)
        x = rng.standard_normal(n)
        # make the last term cancel the others almost exactly
        rest = sum(fr(wi) * fr(xi) for wi, xi in zip(w[:-1], x[:-1]))
        x[-1] = float(-rest / fr(w[-1])) * (1 + 1e-13)
        rel = _check(w, x, parts)
        assert rel < gam_ff(n)


def test_the_bound_is_not_vacuous():
    """The error stays within the bound, and the bound is far below the float32
    path's gamma_n: the stage decides boxes the FP32 pass cannot."""
    rng = np.random.default_rng(3)
    n = 50
    w = rng.standard_normal(n).astype(np.float32)
    x = rng.standard_normal(n)
    rel = _check(w, x, 4)
    assert rel <= gam_ff(n)
    assert gam_ff(n) < 1e-4 * (n * 2.0 ** -24)


def _slice_tree_constant(w, mh, ml, bias, slices):
    """The wide path's layer-1 constant: each slice sums its share of
    w_j (mh_j + ml_j) with exact products and TwoSum (bias in slice 0), then
    the slices' pairs are added in slice order by TwoSum; returns hi + lo
    exactly and sum |fl(w_j mh_j)| as the kernel accumulates it."""
    n = len(w)
    parts = []
    for sl in range(slices):
        s = F32(bias) if sl == 0 else F32(0)
        e = F32(0)
        a = abs(F32(bias)) if sl == 0 else F32(0)
        for j in range(sl, n, slices):
            s, e = ff_mac(w[j], mh[j], ml[j], s, e)
            a = add(a, abs(mul(w[j], mh[j])))
        parts.append((s, e, a))
    s, e, a = parts[0]
    for s1, e1, a1 in parts[1:]:
        t, se = two_sum(s, s1)
        s, e, a = t, add(e, add(e1, se)), add(a, a1)
    hi, lo = two_sum(s, e)
    return fr(hi) + fr(lo), fr(a)


@pytest.mark.parametrize("d", [5, 64, 784])
def test_layer1_constant_slice_tree_within_its_bound(d):
    """2 gamma_{d+2}^2 (1 + gamma_d) sum |p_j| (the bound of the sequential
    compensated chain) also holds for 16 slices merged by TwoSum."""
    rng = np.random.default_rng(d)
    w = rng.standard_normal(d).astype(np.float32)
    m = rng.standard_normal(d)
    mh = m.astype(np.float32)
    ml = (m - mh.astype(np.float64)).astype(np.float32)
    bias = F32(rng.standard_normal())
    got, sabs = _slice_tree_constant(w, mh, ml, bias, 16)
    exact = fr(bias) + sum(fr(wi) * (fr(hi) + fr(lo)) for wi, hi, lo in zip(w, mh, ml))
    g = Fraction((d + 4) * 2.0 ** -24)       # gam<float>(d + 2) = (d + 4) u
    bound = 2 * g * g * sabs * (1 + Fraction((d + 2) * 2.0 ** -24))
    assert abs(got - exact) <= bound
