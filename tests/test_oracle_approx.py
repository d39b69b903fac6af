"""Pins of the approximate counter's oracle (CountingProVe_SLR, Sec. 2.3; Table 1)
against what does not come from its own code (CPU): the published SplitMix64
outputs, the exact count it reduces to without splits, the closed-form unsafe
area of a linear 2-D network (every trial's leaf bracket contains it, and the
2^s-scaled leaf areas average to the root's: the coin is fair and the scale
right), the lower-bound guarantee over many seeds, and the median split."""
import json
import os

import numpy as np

import oracle
from oracle import approx
from workloads import generators as gen

from .pins import _halfplane_area

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.json")


def test_splitmix64_published_outputs():
    for v in json.load(open(GOLDEN))["vectors"]:
        want = [int(x, 0) for x in v["outputs"]]
        got = [int(approx.splitmix64(v["seed"], n)) for n in range(len(want))]
        assert got == want, (v["seed"], got)


def test_draws_are_uniform_and_distinct():
    u = approx.uniform(7, 3, 5, 20000, 4)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    idx = approx.draw_index(3, 5, np.arange(1000)[:, None], np.arange(4)[None, :]).ravel()
    assert np.unique(idx).size == idx.size
    coins = [approx.coin(11, t, j) for t in range(40) for j in range(20)]
    assert 0.4 < np.mean(coins) < 0.6


def test_without_splits_it_is_the_exact_count():
    p = gen.tiny(0)
    r = approx.count_approx(p.net, p.lo, p.hi, p.prop, trials=2, splits=0, leaf_depth=10, beta=1.0, seed=3)
    want = oracle.count(p.net, p.lo, p.hi, p.prop, 10)
    for t in r.trials:
        assert t.splits == 0 and (t.unsafe_lo, t.unsafe_hi) == (want.unsafe_lo, want.unsafe_hi)
        assert t.estimate == want.unsafe_lo / 2 ** 10 and t.volume == 1.0
    assert r.vr_lower == want.unsafe_lo / 2 ** 10 / 2 and r.confidence == 0.75


def _linear_case(seed):
    p = gen.linear_2d(seed, 10)
    w = p.net.W[0][0].astype(np.float64)
    c = float(p.net.b[0][0])
    return p, w, c, _halfplane_area(w, c, (-1.0, -1.0), (1.0, 1.0)) / 4.0


def test_leaf_brackets_contain_the_closed_form_area():
    p, w, c, _ = _linear_case(1)
    for k in range(12):
        t = approx.one_trial(p.net, p.lo, p.hi, p.prop, k, 6, 512, 10, seed=5)
        area = _halfplane_area(w, c, t.leaf_lo.astype(np.float64), t.leaf_hi.astype(np.float64))
        leaf = float(np.prod(t.leaf_hi.astype(np.float64) - t.leaf_lo.astype(np.float64)))
        assert abs(t.volume - leaf / 4.0) <= 1e-15
        assert t.unsafe_lo / 2 ** 10 <= area / leaf + 1e-12 <= t.unsafe_hi / 2 ** 10 + 1e-12
        assert t.estimate <= 2 ** t.splits * area / 4.0 + 1e-12


def _mean_matches_closed_form(seed, scale_shift=0):
    """400 trials on a linear 2-D net: is the mean of 2^(s + scale_shift)
    area(leaf) within 5 standard errors of the closed-form rate?"""
    p, w, c, vr = _linear_case(seed)
    xs = []
    for k in range(400):
        t = approx.one_trial(p.net, p.lo, p.hi, p.prop, k % 64, 5, 256, 0, seed=100 + seed * 1000 + k // 64)
        area = _halfplane_area(w, c, t.leaf_lo.astype(np.float64), t.leaf_hi.astype(np.float64))
        xs.append(2.0 ** (t.splits + scale_shift) * area / 4.0)
    xs = np.array(xs)
    se = xs.std(ddof=1) / np.sqrt(xs.size)
    return abs(xs.mean() - vr) <= 5 * se + 1e-12


def test_scaled_leaf_areas_average_to_the_root_area():
    """E[2^s area(leaf)] = area(root): over 400 trials the mean lies within 5
    standard errors of the closed form."""
    for seed in (0, 2):
        assert _mean_matches_closed_form(seed)


def test_planted_mistakes_fail_the_mean():
    """A coin that always keeps the lower half, or the
    scale 2^(s-1) in place of 2^s, moves the mean away from the closed form."""
    assert not _mean_matches_closed_form(0, scale_shift=-1)
    orig = approx.coin
    try:
        approx.coin = lambda seed, trial, split: 0       # always the lower half
        assert not _mean_matches_closed_form(0) or not _mean_matches_closed_form(2)
    finally:
        approx.coin = orig


def test_lower_bound_holds_with_its_confidence():
    """Over 60 seeds with beta = 1 and 2 trials (confidence 3/4), the lower
    bound exceeds the closed-form rate in at most 3/4 of the binomial slack."""
    p, w, c, vr = _linear_case(3)
    above = 0
    n = 60
    for s in range(n):
        r = approx.count_approx(p.net, p.lo, p.hi, p.prop, trials=2, splits=4, samples=256, leaf_depth=8, beta=1.0,
                                seed=s)
        above += r.vr_lower > vr
    # P(above) <= 1/4: 60 runs exceed it by 5 sigma only with probability ~1e-6
    assert above <= 0.25 * n + 5 * np.sqrt(n * 0.25 * 0.75)


def test_split_point_is_the_lower_median_of_the_violations():
    p = gen.acas_shaped(0)
    t = approx.one_trial(p.net, p.lo, p.hi, p.prop, 0, 3, 2048, 4, seed=9)
    lo = p.lo.astype(np.float32).copy()
    hi = p.hi.astype(np.float32).copy()
    for j, (i, m, cn) in enumerate(zip(t.dims, t.points, t.coins)):
        assert i == int(np.argmax(hi.astype(np.float64) - lo.astype(np.float64)))
        u = approx.uniform(9, 0, j, 2048, p.d)
        x = lo.astype(np.float64) + (hi.astype(np.float64) - lo.astype(np.float64)) * u
        v = np.sort(x[oracle.unsafe_points(p.net, p.prop, x), i])
        if v.size:
            # as many sampled violations on each side of the split, up to one
            below = int(np.count_nonzero(v < m))
            assert abs(below - (v.size - below)) <= 2, (below, v.size)
            assert m == np.float32(v[(v.size - 1) // 2])
        if cn == 0:
            hi[i] = m
        else:
            lo[i] = m
    assert np.array_equal(lo, t.leaf_lo) and np.array_equal(hi, t.leaf_hi)


def test_ties_split_the_lowest_index():
    """The widest side, ties to the lowest index: on the square root box of
    the linear 2-D case the first split is along x_0, the second along x_1
    (x_0 is then half as wide), and so on alternately."""
    p, _, _, _ = _linear_case(1)
    t = approx.one_trial(p.net, p.lo, p.hi, p.prop, 0, 6, 256, 0, seed=5)
    assert t.dims == [0, 1, 0, 1, 0, 1][:len(t.dims)] and len(t.dims) >= 2
