"""The oracle's gradient split rule and per-box bisection against hand-worked
values, closed forms and sampling (CPU only)."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen
from workloads.generators import Network, Problem, Property


def _prop(rows_per_clause, C, e, strict=None):
    C = np.asarray(C, dtype=np.float32)
    R = C.shape[0]
    return Property(np.asarray(rows_per_clause, dtype=np.int32), C, np.asarray(e, dtype=np.float32),
                    np.zeros(R, dtype=np.uint8) if strict is None else np.asarray(strict, dtype=np.uint8))


def test_decision_weights_hand_worked():
    # two clauses: rows {0, 1} and {2}
    prop = _prop([2, 1], np.eye(3), np.zeros(3))
    # safe gap 0.5 + 1 = 1.5 <= unsafe gap min(2, 3) = 2: towards SAFE, the
    # smallest hi of each clause that is still positive
    w_hi, w_lo, M = oracle.decision_weights(np.array([-1.0, -2.0, -3.0]), np.array([2.0, 0.5, 1.0]), prop)
    assert M == 1.5 and list(w_hi) == [0, 1, 1] and list(w_lo) == [0, 0, 0]
    # safe gap 3 + 2 = 5 > unsafe gap min(0.3, 5) = 0.3: towards UNSAFE through
    # the lowest lo of the first clause
    w_hi, w_lo, M = oracle.decision_weights(np.array([-0.1, -0.3, -5.0]), np.array([4.0, 3.0, 2.0]), prop)
    assert M == pytest.approx(0.3) and list(w_hi) == [0, 0, 0] and list(w_lo) == [0, -1, 0]
    # clause 0 already excluded (hi_0 < 0) adds nothing to the safe gap (2);
    # unsafe gaps tie at 1: the first clause, and its first lowest row
    w_hi, w_lo, M = oracle.decision_weights(np.array([-1.0, -1.0, -1.0]), np.array([-0.5, 1.0, 2.0]), prop)
    assert M == 1.0 and list(w_lo) == [-1, 0, 0] and list(w_hi) == [0, 0, 0]
    # nothing left to gain: the box is decided SAFE, M = 0 and no weight
    w_hi, w_lo, M = oracle.decision_weights(np.array([-3.0, -3.0, -3.0]), np.array([-0.5, 1.0, -2.0]), prop)
    assert M == 0.0 and not w_hi.any() and not w_lo.any()


def _affine_problem(seed, d=6):
    rng = np.random.default_rng(seed)
    W = rng.normal(size=(1, d)).astype(np.float32)
    b = np.array([0.3], dtype=np.float32)
    lo = rng.uniform(-1, 0, size=d).astype(np.float32)
    hi = (lo + rng.uniform(0.1, 1.0, size=d)).astype(np.float32)
    prop = _prop([1], [[-1.0]], [0.0])          # unsafe: y <= 0
    return Network([W], [b]), lo, hi, prop, W[0].astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radius_gradient_of_an_affine_map_is_abs_weight(seed):
    """Row -(w.x + b) over a box: lo = -(w.m + b) - |w|.r, hi = -(w.m + b) + |w|.r, so
    dM/dr_i = |w_i| in both directions of the loss."""
    net, lo, hi, prop, w = _affine_problem(seed)
    g = oracle.radius_gradient(net, lo, hi, prop)
    np.testing.assert_allclose(g, np.abs(w), rtol=1e-9, atol=1e-9)
    S = oracle.split_set(net, lo, hi, prop, k=3)
    width = hi.astype(np.float64) - lo.astype(np.float64)
    want = np.sort(np.argsort(-(np.abs(w) * width), kind="stable")[:3])
    assert list(S) == list(want)
    dims = oracle.gradient_split(net, prop, S)(0, np.zeros(1, dtype=np.int64), lo[None].astype(np.float64),
                                               hi[None].astype(np.float64))
    assert dims[0] == S[int(np.argmax(np.abs(w[S]) * width[S]))]


def test_radius_gradient_through_active_relus():
    """Every ReLU active on the box: the network is the affine map W2 W1, and
    dM/dr_i = |(c W2 W1)_i|."""
    rng = np.random.default_rng(4)
    W1 = rng.normal(size=(5, 3)).astype(np.float32)
    b1 = np.full(5, 20.0, dtype=np.float32)
    W2 = rng.normal(size=(2, 5)).astype(np.float32)
    b2 = np.zeros(2, dtype=np.float32)
    net = Network([W1, W2], [b1, b2])
    prop = _prop([1], [[1.0, -1.0]], [0.0])
    lo = np.array([-0.5, -0.2, 0.1], dtype=np.float32)
    hi = np.array([0.5, 0.3, 0.4], dtype=np.float32)
    g = oracle.radius_gradient(net, lo, hi, prop)
    w_eff = np.array([1.0, -1.0]) @ W2.astype(np.float64) @ W1.astype(np.float64)
    np.testing.assert_allclose(g, np.abs(w_eff), rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("name,D", [("tiny", 12), ("acas", 8), ("rare", 10)])
def test_per_box_bisection_reproduces_the_schedule(name, D):
    """Splitting each box along the level's widest-side dimension gives the
    scheduled count, level by level and leaf by leaf."""
    p = gen.make(name)
    sched = oracle.split_schedule(p.lo, p.hi, D)
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True)
    got = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True,
                       split=lambda t, paths, lo, hi: np.full(paths.shape[0], sched[t]))
    assert (got.unsafe_lo, got.unsafe_hi) == (want.unsafe_lo, want.unsafe_hi)
    assert got.levels == want.levels
    assert sorted(got.leaves) == sorted(want.leaves)
    # the leaf boxes are the decoded ones
    lo, hi = oracle.decode(np.array([c for c, t, _ in got.leaves if t == D]), D, sched, p.lo, p.hi)
    blo = np.array([b[0] for (c, t, _), b in zip(got.leaves, got.leaf_boxes) if t == D])
    if blo.size:
        assert np.array_equal(lo, blo)


def test_gradient_rule_count_is_sound_and_tiles_the_box():
    p = gen.make("tiny")
    D = 12
    S = oracle.split_set(p.net, p.lo, p.hi, p.prop)
    assert list(S) == [0, 1]
    r = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True,
                     split=oracle.gradient_split(p.net, p.prop, S))
    # the leaves partition the root box: their volumes add up to 2^D units
    assert sum(1 << (D - t) for _, t, _ in r.leaves) == 1 << D
    vol = sum(np.prod((hi - lo) / (p.hi.astype(np.float64) - p.lo)) for lo, hi in r.leaf_boxes)
    assert vol == pytest.approx(1.0, abs=1e-12)
    # decided leaves hold only unsafe (UNSAFE) or only safe (SAFE) points
    rng = np.random.default_rng(0)
    for (_, t, cl), (lo, hi) in zip(r.leaves, r.leaf_boxes):
        if cl == oracle.UNDECIDED:
            continue
        x = lo + (hi - lo) * rng.random((64, p.d))
        u = oracle.unsafe_points(p.net, p.prop, x)
        assert u.all() if cl == oracle.UNSAFE else not u.any()
    # the bracket holds the sampled violation rate (6 sigma)
    n = 200_000
    x = p.lo + (p.hi - p.lo) * rng.random((n, p.d))
    f = oracle.unsafe_points(p.net, p.prop, x).mean()
    sig = np.sqrt(max(f * (1 - f), 1e-12) / n)
    assert r.unsafe_lo / 2 ** D - 6 * sig <= f <= r.unsafe_hi / 2 ** D + 6 * sig
