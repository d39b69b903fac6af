"""Pins of the oracle's relaxation of S-shaped activations (tanh, logistic
sigmoid) against values that do not come from its code (CPU): hand-derived
bounds of tanh(x) - tanh(x) (identically 0) in the straddling, concave and
convex cases, dense sampling inside the bounds of the tanh- and sigmoid-
network workloads, and the Moore-interval image of a monotone function."""
import math

import numpy as np
import pytest

import oracle
from oracle import slr as oslr
from workloads import generators as gen


def _twin(lo, hi, act="tanh"):
    """y = s(x) - s(x) with both neurons on z = x: the SLR bound is the gap
    between the upper line of the first and the lower line of the second."""
    net = gen.Network([np.array([[1.0], [1.0]], np.float32), np.array([[1.0, -1.0]], np.float32)],
                      [np.zeros(2, np.float32), np.zeros(1, np.float32)], act=[act])
    lo_, hi_, _ = oracle.slr_forward(net, np.array([lo]), np.array([hi]))
    return float(lo_[0]), float(hi_[0])


def _dt(z):
    return 1.0 - math.tanh(z) ** 2


def test_straddling_interval_uses_the_smaller_end_slope():
    l, u = -1.0, 2.0
    lam = min(_dt(l), _dt(u))                      # = 1 - tanh(2)^2
    # U = lam z + tanh(u) - lam u, L = lam z + tanh(l) - lam l: the z terms cancel
    want = math.tanh(u) - lam * u - (math.tanh(l) - lam * l)
    lo, hi = _twin(l, u)
    assert abs(hi - want) < 1e-14 and abs(lo + want) < 1e-14


def test_concave_interval_tangent_above_chord_below():
    l, u = 0.5, 2.0
    m = 0.5 * (l + u)
    s = (math.tanh(u) - math.tanh(l)) / (u - l)
    up = lambda z: _dt(m) * (z - m) + math.tanh(m)          # noqa: E731  tangent at the midpoint
    dn = lambda z: s * (z - l) + math.tanh(l)                 # noqa: E731  chord
    want = max(up(z) - dn(z) for z in (l, u))               # linear in z: an end point
    lo, hi = _twin(l, u)
    assert abs(hi - want) < 1e-14 and abs(lo + want) < 1e-14
    assert want > 0


def test_convex_interval_chord_above_tangent_below():
    l, u = -2.5, -0.25
    m = 0.5 * (l + u)
    s = (math.tanh(u) - math.tanh(l)) / (u - l)
    up = lambda z: s * (z - l) + math.tanh(l)                 # noqa: E731  chord
    dn = lambda z: _dt(m) * (z - m) + math.tanh(m)          # noqa: E731  tangent
    want = max(up(z) - dn(z) for z in (l, u))
    lo, hi = _twin(l, u)
    assert abs(hi - want) < 1e-14 and abs(lo + want) < 1e-14


def test_sigmoid_straddling_case():
    sg = lambda z: 1.0 / (1.0 + math.exp(-z))                # noqa: E731
    ds = lambda z: sg(z) * (1.0 - sg(z))                      # noqa: E731
    l, u = -3.0, 0.5
    lam = min(ds(l), ds(u))
    want = sg(u) - lam * u - (sg(l) - lam * l)
    lo, hi = _twin(l, u, "sigmoid")
    assert abs(hi - want) < 1e-14 and abs(lo + want) < 1e-14


def test_zero_width_box_gives_the_value():
    lo, hi = _twin(0.7, 0.7)
    assert lo == 0.0 and hi == 0.0


@pytest.mark.parametrize("name", ["acas_tanh", "nav_sigmoid"])
def test_sampled_points_lie_inside(name):
    p = gen.make(name)
    rng = np.random.default_rng(4)
    for k in range(6):
        u = np.sort(rng.random((2, p.d)), axis=0)
        lo = p.lo + (p.hi - p.lo) * u[0]
        hi = p.lo + (p.hi - p.lo) * u[1]
        if k == 0:
            lo, hi = p.lo.astype(np.float64), p.hi.astype(np.float64)
        rl, rh, _ = oracle.slr_forward(p.net, lo[None], hi[None], p.prop)
        x = lo + (hi - lo) * rng.random((20000, p.d))
        rows, _ = oracle.forward_points(p.net, x, p.prop)
        scale = np.abs(rows).max() + 1.0
        assert np.all(rows >= rl[0] - 1e-12 * scale) and np.all(rows <= rh[0] + 1e-12 * scale), (name, k)


def test_interval_image_of_a_monotone_activation():
    net = gen.Network([np.array([[2.0]], np.float32), np.array([[1.0]], np.float32)],
                      [np.array([0.5], np.float32), np.zeros(1, np.float32)], act=["sigmoid"])
    lo, hi, _ = oracle.interval_forward(net, np.array([[-1.0]]), np.array([[0.25]]))
    sg = lambda z: 1.0 / (1.0 + math.exp(-z))                # noqa: E731
    assert abs(lo[0, 0] - sg(-1.5)) < 1e-15 and abs(hi[0, 0] - sg(1.0)) < 1e-15


def test_swapped_concave_rule_is_caught():
    """A planted mistake (tangent and chord swapped on the concave side) puts
    the value 0 of tanh(x) - tanh(x) outside its bounds."""
    orig = oslr._relax_s

    def swapped(U, L, ll, uu, name):
        U2, L2 = orig(U, L, ll, uu, name)
        conc = ll >= 0
        U3 = np.where(conc[..., None], L2 * 0 + L2, U2)     # chord as the upper line
        L3 = np.where(conc[..., None], U2 * 0 + U2, L2)     # tangent as the lower line
        return U3, L3
    oslr._relax_s = swapped
    try:
        lo, hi = _twin(0.5, 2.0)
    finally:
        oslr._relax_s = orig
    assert not (lo <= 0.0 <= hi)
