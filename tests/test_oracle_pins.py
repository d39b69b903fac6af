"""The FP64 oracle against brute force, closed forms and hand-worked examples (CPU only)."""
import numpy as np
import pytest

import oracle
from oracle import slr as oslr
from workloads import generators as gen

from . import pins


def test_concretize_matches_box_vertices():
    pins.check_concretize_vertices()


def test_hand_worked_bounds(golden):
    pins.check_hand_bounds(golden)


def test_hand_worked_classification(golden):
    pins.check_hand_classify(golden)


def test_hand_worked_schedule_and_decode(golden):
    pins.check_hand_schedule(golden)


def test_hand_worked_counts(golden):
    pins.check_hand_count(golden)


def test_exact_where_every_relu_is_stable():
    pins.check_exact_on_stable_region()


def test_affine_network_is_exact():
    pins.check_affine_net_exact()


@pytest.mark.parametrize("mode", ["neurify", "paper_literal"])
def test_soundness_by_sampling(mode):
    probs = [gen.tiny(0), gen.acas_shaped(0), gen.nav_shaped(0), gen.rare_violation(0)]
    pins.check_soundness_sampling(probs, n_points=20000, n_boxes=5, mode=mode)


def test_soundness_million_points_tiny_root():
    """10^6 sampled points of the 2-D workload lie inside the root bounds."""
    pins.check_soundness_sampling([gen.tiny(0)], n_points=1_000_000, n_boxes=0)


def test_soundness_full_grid_2d():
    pins.check_grid_2d(gen.tiny(0))
    pins.check_grid_2d(gen.tiny(7))


def test_count_linear_2d_closed_form():
    pins.check_count_linear_2d()


def test_count_single_layer_1d_closed_form():
    pins.check_count_1d()


def test_leaves_agree_with_sampling():
    pins.check_leaves_by_sampling(gen.tiny(0), 10)


def test_count_brackets_monte_carlo():
    """The MC unsafe fraction over 10^6 points lies in [lo, hi] / 2^D up to 6 sigma."""
    p = gen.tiny(0)
    r = oracle.count(p.net, p.lo, p.hi, p.prop, p.depth)
    rng = np.random.default_rng(99)
    n = 1_000_000
    x = p.lo + (p.hi - p.lo) * rng.random((n, p.d))
    f = float(np.mean(oracle.unsafe_points(p.net, p.prop, x)))
    sig = np.sqrt(max(f * (1 - f), 1e-12) / n)
    assert r.unsafe_lo / 2 ** p.depth - 6 * sig <= f <= r.unsafe_hi / 2 ** p.depth + 6 * sig


def test_count_bracket_narrows_with_depth():
    """Deeper counts refine shallower ones: [lo, hi] / 2^D is nested as D grows."""
    p = gen.tiny(0)
    prev = None
    for D in (4, 6, 8, 10, 12):
        r = oracle.count(p.net, p.lo, p.hi, p.prop, D)
        lo, hi = r.unsafe_lo / 2 ** D, r.unsafe_hi / 2 ** D
        if prev is not None:
            assert prev[0] <= lo and hi <= prev[1]
        prev = (lo, hi)


def test_exact_rationals_agree_with_float64():
    """Every step is rational: the oracle in exact Fractions classifies as in FP64."""
    p = gen.tiny(0)
    D = 6
    sched = oracle.split_schedule(p.lo, p.hi, D)
    codes = np.arange(1 << D)
    a64, b64 = oracle.decode(codes, D, sched, p.lo, p.hi)
    lo64, hi64, _ = oracle.slr_forward(p.net, a64, b64, p.prop)
    net_x, prop_x, _, _ = oracle.to_exact(p.net, p.prop, p.lo, p.hi)
    from fractions import Fraction
    fr = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])
    lox, hix, _ = oracle.slr_forward(net_x, fr(a64), fr(b64), prop_x, exact=True)
    err = np.max(np.abs(np.array(lox - fr(lo64), dtype=np.float64)))
    err = max(err, np.max(np.abs(np.array(hix - fr(hi64), dtype=np.float64))))
    assert err < 1e-12
    c64 = oracle.classify(lo64, hi64, p.prop)
    cx = oracle.classify(lox, hix, prop_x)
    assert np.array_equal(c64, cx)


def test_first_hidden_layer_equals_intervals():
    """Before any relaxation, SLR and Moore intervals give the same pre-activation bounds."""
    p = gen.acas_shaped(0)
    _, _, pre_s = oracle.slr_forward(p.net, p.lo, p.hi, p.prop)
    _, _, pre_i = oracle.interval_forward(p.net, p.lo, p.hi, p.prop)
    np.testing.assert_allclose(pre_s[0][0], pre_i[0][0], atol=1e-12)
    np.testing.assert_allclose(pre_s[0][3], pre_i[0][1], atol=1e-12)


def test_slr_is_not_always_inside_intervals(golden):
    """SLR's lower relaxation can go below 0 where an interval would clip: a worked counterexample."""
    ex = [e for e in golden["bounds"] if e["name"] == "identity_via_two_relus"][0]
    assert ex["neurify"][0][0] < ex["interval"][0][0]


def test_slr_tighter_than_intervals_on_workloads():
    """On the paper-shaped workloads SLR row bounds are (much) tighter than intervals."""
    for p in (gen.acas_shaped(0), gen.nav_shaped(0)):
        lo_s, hi_s, _ = oracle.slr_forward(p.net, p.lo, p.hi, p.prop)
        lo_i, hi_i, _ = oracle.interval_forward(p.net, p.lo, p.hi, p.prop)
        assert np.sum(hi_s - lo_s) < np.sum(hi_i - lo_i)


def test_children_partition_parent():
    """The two children of a box split one side at its midpoint and nothing else."""
    p = gen.acas_shaped(0)
    D = 9
    sched = oracle.split_schedule(p.lo, p.hi, D)
    for t in range(D):
        codes = np.arange(min(1 << t, 64))
        lo, hi = oracle.decode(codes, t, sched, p.lo, p.hi)
        clo, chi = oracle.decode(np.concatenate([2 * codes, 2 * codes + 1]), t + 1, sched, p.lo, p.hi)
        n = codes.shape[0]
        i = sched[t]
        for side in range(2):
            cl, ch = clo[side * n:(side + 1) * n], chi[side * n:(side + 1) * n]
            other = np.arange(p.d) != i
            assert np.array_equal(cl[:, other], lo[:, other]) and np.array_equal(ch[:, other], hi[:, other])
        mid = (lo[:, i] + hi[:, i]) / 2
        assert np.array_equal(clo[:n, i], lo[:, i]) and np.array_equal(chi[:n, i], mid)
        assert np.array_equal(clo[n:, i], mid) and np.array_equal(chi[n:, i], hi[:, i])


def test_interval_count_never_beats_slr_on_tiny():
    """The naive-interval counter (the paper's Exact Count baseline) decides no more volume."""
    p = gen.tiny(0)
    rs = oracle.count(p.net, p.lo, p.hi, p.prop, 12)
    ri = oracle.count(p.net, p.lo, p.hi, p.prop, 12, bound="interval")
    assert ri.unsafe_lo <= ri.unsafe_hi and rs.unsafe_lo <= rs.unsafe_hi
    # both brackets contain the MC rate
    rng = np.random.default_rng(5)
    x = p.lo + (p.hi - p.lo) * rng.random((200000, 2))
    f = float(np.mean(oracle.unsafe_points(p.net, p.prop, x)))
    s = 6 * np.sqrt(f * (1 - f) / 200000)
    for r in (rs, ri):
        assert r.unsafe_lo / 4096 - s <= f <= r.unsafe_hi / 4096 + s
    assert (rs.unsafe_hi - rs.unsafe_lo) <= (ri.unsafe_hi - ri.unsafe_lo)


def test_relaxation_lines_touch_relu_at_the_ends():
    """Upper chord meets relu at both ends of [lu, uu]; lower slope passes through 0."""
    U = np.array([[[2.0, -1.0]]])   # 2x - 1 on [0, 1]: lu = -1, uu = 1
    L = np.array([[[2.0, -1.5]]])   # 2x - 1.5: ll = -1.5, ul = 0.5
    a, b = np.zeros((1, 1)), np.ones((1, 1))
    ll, ul = oracle.concretize(L, a, b)
    lu, uu = oracle.concretize(U, a, b)
    U2, L2 = oslr._relax(U, L, ll, ul, lu, uu, None, "neurify")
    assert abs(U2[0, 0, 0] * 0.0 + U2[0, 0, 1] - 0.0) < 1e-15      # chord at lu is 0
    assert abs(U2[0, 0, 0] * 1.0 + U2[0, 0, 1] - 1.0) < 1e-15      # chord at uu is uu
    assert abs(L2[0, 0, 0] * 0.75 + L2[0, 0, 1]) < 1e-15          # alpha L vanishes where L does


def test_slope_gradient_hand_worked():
    """abs_via_two_relus with slopes a1, a2: lo = min_x (a1 - a2) x on [-1, 1] = -|a1 - a2|."""
    from workloads.generators import Network
    net = Network([np.array([[1.0], [-1.0]], np.float32), np.array([[1.0, 1.0]], np.float32)],
                  [np.zeros(2, np.float32), np.zeros(1, np.float32)])
    alpha = [np.array([0.7, 0.2])]
    J = oracle.objective(net, np.array([-1.0]), np.array([1.0]), None, alpha, np.array([0.0]), np.array([1.0]))
    assert abs(J + 0.5) < 1e-12
    g = oracle.fd_gradients(net, np.array([-1.0]), np.array([1.0]), None, alpha, np.array([0.0]), np.array([1.0]))
    np.testing.assert_allclose(g["alpha"][0], [-1.0, 1.0], atol=1e-7)


def test_box_gradient_of_an_affine_network_closed_form():
    """One affine layer y = w.x + c: hi = w.m + c + |w|.r, so dhi/dlo_j = (w_j - |w_j|)/2, dhi/dhi_j = (w_j + |w_j|)/2."""
    from workloads.generators import Network
    rng = np.random.default_rng(4)
    w = rng.normal(size=(1, 4)).astype(np.float32)
    net = Network([w], [np.array([0.3], np.float32)])
    lo = rng.uniform(-1, 0, 4)
    hi = lo + rng.uniform(0.2, 1, 4)
    g = oracle.fd_gradients(net, lo, hi, None, [], np.array([1.0]), np.array([0.0]))
    wd = w[0].astype(np.float64)
    np.testing.assert_allclose(g["lo"], (wd - np.abs(wd)) / 2, atol=1e-7)
    np.testing.assert_allclose(g["hi"], (wd + np.abs(wd)) / 2, atol=1e-7)
    # weight gradient: d hi / d w_j = m_j + sign(w_j) r_j
    np.testing.assert_allclose(g["W"][0][0], (lo + hi) / 2 + np.sign(wd) * (hi - lo) / 2, atol=1e-7)


def test_default_slope_box_gradient_closed_form():
    """x -> relu(x) on [l, u], l < 0 < u: lo = u l / (u - l) (slope u/(u-l) on L = x), hi = u (chord)."""
    from workloads.generators import Network
    net = Network([np.array([[1.0]], np.float32), np.array([[1.0]], np.float32)],
                  [np.zeros(1, np.float32), np.zeros(1, np.float32)])
    l, u = -0.75, 1.25
    g = oracle.fd_gradients(net, np.array([l]), np.array([u]), None, None, np.array([0.0]), np.array([1.0]))
    np.testing.assert_allclose(g["lo"], [u * u / (u - l) ** 2], atol=1e-7)
    np.testing.assert_allclose(g["hi"], [-l * l / (u - l) ** 2], atol=1e-7)
    g = oracle.fd_gradients(net, np.array([l]), np.array([u]), None, None, np.array([1.0]), np.array([0.0]))
    np.testing.assert_allclose(g["lo"], [0.0], atol=1e-7)
    np.testing.assert_allclose(g["hi"], [1.0], atol=1e-7)
