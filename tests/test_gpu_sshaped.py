"""Networks with S-shaped activations (tanh, logistic sigmoid) through the C
ABI against the FP64 oracle (needs a GB300): bounds sound and within the
bound tolerance on every path, a million sampled points inside, counts
bit-exact (FP64 re-check included), interval mode, the tensor-core and wide
paths, the approximate counter, and the refusal of slope features."""
import numpy as np
import pytest

import oracle
from oracle import approx
from workloads import generators as gen

from .gpu_common import bound_errors, random_sub_boxes
from .test_gpu_parity import _check_count

pytestmark = pytest.mark.gpu

CONFIGS = ["acas_tanh", "nav_sigmoid", "tiny_tanh", "tiny_sigmoid"]

# The FP32 path evaluates tanh and exp in float (2 ulp): the lines' slopes and
# values carry about 2^-21 absolutely, which a tangent's intercept multiplies
# by the pre-activation midpoint |m| (up to about 10 here) and each row sums
# over 50-64 neurons; against row scales of 1-10 that is a few 1e-5, so the
# raw bounds of these networks are held to 4e-5 of the row scale (ReLU
# networks: 1e-5).  The widened bounds contain the oracle's exactly.
SSHAPE_RTOL = 4e-5


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _bounds(pkg, p, lo, hi, **opt):
    with pkg.Counter(0) as c:
        c.set_problem(p)
        if opt:
            c.set_options(**opt)
        return c.bounds(lo, hi, want_err=True)


@pytest.mark.parametrize("name", CONFIGS)
@pytest.mark.parametrize("n", [1, 37, 700])
@pytest.mark.parametrize("path", ["fp32", "tf32", "wide"])
def test_bounds_match_oracle(pkg, name, n, path):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, n, seed=n + 3)
    opt = {"fp32": {}, "tf32": {"precision": pkg.PREC_TC_TF32}, "wide": {"wide": 1}}[path]
    rl, rh, cls, err = _bounds(pkg, p, lo, hi, **opt)
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= SSHAPE_RTOL and ehi.max() <= SSHAPE_RTOL, (elo.max(), ehi.max())
    ocls = oracle.classify(olo, ohi, p.prop)
    dec = cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], ocls[dec])


@pytest.mark.parametrize("name", CONFIGS)
def test_a_million_points_inside(pkg, name):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, 16, seed=21)
    lo[0], hi[0] = p.lo, p.hi
    rl, rh, _, _ = _bounds(pkg, p, lo, hi)
    rng = np.random.default_rng(5)
    for k in range(16):
        x = lo[k].astype(np.float64) + (hi[k].astype(np.float64) - lo[k]) * rng.random((1_000_000 // 16, p.d))
        rows, _ = oracle.forward_points(p.net, x, p.prop)
        assert np.all(rows >= rl[k]) and np.all(rows <= rh[k]), k


@pytest.mark.parametrize("name,D", [("tiny_tanh", 16), ("tiny_sigmoid", 16), ("acas_tanh", 11), ("nav_sigmoid", 9)])
def test_count_matches_oracle(pkg, name, D):
    """Counts, per-level statistics and leaf sets bit-exact.  The tiny-shaped
    networks decide boxes from the first levels on; the ACAS- and nav-shaped
    ones decide nothing at these depths (their S-shaped bounds tighten only
    for boxes about 1 % of the root's side) and check the per-level totals."""
    got = _check_count(pkg, gen.make(name), D)
    assert got["tie_leaves"] == 0
    if name.startswith("tiny"):
        assert sum(got["level_safe"]) > 0 and sum(got["level_unsafe"]) > 0


@pytest.mark.parametrize("name,D", [("tiny_tanh", 14), ("tiny_sigmoid", 14), ("acas_tanh", 10), ("nav_sigmoid", 8)])
def test_interval_mode_count_matches_oracle(pkg, name, D):
    p = gen.make(name)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(relax_mode=2)
        got = c.count(D)
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D, bound="interval")
    assert (got["unsafe_lo"], got["unsafe_hi"]) == (want.unsafe_lo, want.unsafe_hi)
    assert got["boxes"] == want.boxes


@pytest.mark.parametrize("name", ["tiny_tanh", "tiny_sigmoid"])
def test_tensor_core_and_wide_counts(pkg, name):
    p = gen.make(name)
    D = 14
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D)
    for opt in (dict(precision=pkg.PREC_TC_TF32), dict(wide=1)):
        with pkg.Counter(0) as c:
            c.set_problem(p)
            c.set_options(**opt)
            r = c.count(D)
        assert r["unsafe_lo"] <= want.unsafe_lo <= want.unsafe_hi <= r["unsafe_hi"], opt
        if r["tie_leaves"] == 0:
            assert (r["unsafe_lo"], r["unsafe_hi"]) == (want.unsafe_lo, want.unsafe_hi), opt


@pytest.mark.parametrize("name", ["tiny_tanh", "acas_tanh"])
def test_approximate_counter_matches_oracle(pkg, name):
    p = gen.make(name)
    kw = dict(trials=3, splits=6, samples=2048, leaf_depth=8, beta=1.0, seed=4)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        got = c.count_approx(**kw)
    want = approx.count_approx(p.net, p.lo, p.hi, p.prop, **kw)
    for t, w in enumerate(want.trials):
        assert np.array_equal(got["leaf_lo"][t], w.leaf_lo) and np.array_equal(got["leaf_hi"][t], w.leaf_hi)
        assert (got["leaf_unsafe_lo"][t], got["leaf_unsafe_hi"][t]) == (w.unsafe_lo, w.unsafe_hi)
    assert got["vr_lower"] == want.vr_lower


def test_slope_features_are_refused(pkg):
    p = gen.make("acas_tanh")
    lo, hi = random_sub_boxes(p, 4, seed=1)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(alpha_steps=5)
        with pytest.raises(pkg.SlrError) as ei:
            c.count(8)
        assert ei.value.code == -7
        c.set_options()
        R = p.prop.C.shape[0]
        with pytest.raises(pkg.SlrError) as ei:
            c.margin_backward(lo, hi, np.ones((4, R), np.float32), np.ones((4, R), np.float32))
        assert ei.value.code == -7
        with pytest.raises(pkg.SlrError) as ei:
            c.bounds(lo, hi, alpha=np.full((4, c.alpha_width()), 0.5, np.float32))
        assert ei.value.code == -7


def test_activation_arguments(pkg):
    from paper_2312_05890_gb300 import slr_set_activations
    p = gen.make("acas")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        for bad in (["tanh"] * 3, [7] * (p.net.K - 1)):
            with pytest.raises(pkg.SlrError) as ei:
                slr_set_activations(c.ctx, bad)
            assert ei.value.code == -1
        relu = c.count(10)
        slr_set_activations(c.ctx, ["relu"] * (p.net.K - 1))
        assert c.count(10)["unsafe_hi"] == relu["unsafe_hi"]
