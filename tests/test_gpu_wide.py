"""The wide path (per-box state in GPU memory, one tensor-core product per
layer) against the FP64 oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen

from .gpu_common import BOUND_RTOL, bound_errors, random_sub_boxes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _counter(pkg, p, **opt):
    c = pkg.Counter(0)
    c.set_problem(p)
    c.set_options(**opt)
    return c


def _check_bounds(p, lo, hi, rl, rh, cls, err):
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale), "wide lower bound above the exact SLR bound"
    assert np.all(rh >= ohi - 1e-12 * scale), "wide upper bound below the exact SLR bound"
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL, (elo.max(), ehi.max())
    ocls = oracle.classify(olo, ohi, p.prop)
    dec = cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], ocls[dec])


@pytest.mark.parametrize("name", ["tiny", "acas", "nav"])
@pytest.mark.parametrize("n", [1, 37, 700])
def test_wide_bounds_match_oracle(pkg, name, n):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, n, seed=n + 11)
    with _counter(pkg, p, wide=1) as c:
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    _check_bounds(p, lo, hi, rl, rh, cls, err)


def test_wide_and_tile_paths_agree(pkg):
    """Both paths bound the same float32 network: their FP32 SLR bounds agree closely."""
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 500, seed=5)
    with _counter(pkg, p) as c:
        a = c.bounds(lo, hi, want_err=True)
    with _counter(pkg, p, wide=1) as c:
        b = c.bounds(lo, hi, want_err=True)
    scale = np.maximum(np.abs(a[0]), np.abs(a[1])) + (a[1] - a[0])
    assert np.max(np.abs((a[0] + a[3]) - (b[0] + b[3])) / scale) <= 2 * BOUND_RTOL
    assert np.max(np.abs((a[1] - a[3]) - (b[1] - b[3])) / scale) <= 2 * BOUND_RTOL


@pytest.mark.parametrize("name,D", [("tiny", 16), ("acas", 11), ("nav", 9), ("acas", 16)])
def test_wide_count_equals_oracle(pkg, name, D):
    """The wide path's boxes whose class depends on its widening are re-bounded
    by the FP64 tile kernel (these networks fit it): counts, per-level
    statistics and leaf sets equal the oracle's."""
    p = gen.make(name)
    with _counter(pkg, p, wide=1, record_leaves=1) as c:
        r = c.count(D)
        codes, depth, cls = c.leaves()
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True)
    assert r["tie_leaves"] == 0
    assert (r["unsafe_lo"], r["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
    for t, lv in enumerate(ref.levels):
        assert (r["level_boxes"][t], r["level_safe"][t], r["level_unsafe"][t], r["level_undecided"][t]) == \
            (lv["boxes"], lv["safe"], lv["unsafe"], lv["undecided"]), t
    assert sorted(zip(codes.tolist(), depth.tolist(), cls.tolist())) == sorted(ref.leaves)
    if name == "acas" and D == 16:
        assert r["rechecked"] > 0


def test_wide_count_without_recheck_brackets_oracle(pkg):
    """With the re-check off, boxes whose class depends on the widening stay
    undecided (tie_leaves): the bracket contains the oracle's."""
    p = gen.make("acas")
    with _counter(pkg, p, wide=1, fp64_recheck=0) as c:
        r = c.count(14)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, 14)
    assert r["unsafe_lo"] <= ref.unsafe_lo <= ref.unsafe_hi <= r["unsafe_hi"]


def test_mnist_shaped_bounds(pkg):
    """784 -> 3x256 -> 10: sampled boxes agree with the oracle; sampled points lie inside."""
    p = gen.make("mnist")
    lo, hi = random_sub_boxes(p, 6, seed=2, min_frac=0.5)
    lo = np.vstack([p.lo[None], lo]).astype(np.float32)
    hi = np.vstack([p.hi[None], hi]).astype(np.float32)
    with _counter(pkg, p) as c:
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    _check_bounds(p, lo, hi, rl, rh, cls, err)
    rng = np.random.default_rng(0)
    for b in range(len(lo)):
        x = lo[b] + (hi[b] - lo[b]) * rng.random((2000, p.d))
        y = oracle.forward_points(p.net, x, p.prop)[0]
        assert np.all(y >= rl[b]) and np.all(y <= rh[b])


def test_mnist_shaped_count_small_depth(pkg):
    p = gen.make("mnist")
    with _counter(pkg, p) as c:
        r = c.count(4)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, 4)
    assert r["unsafe_lo"] <= ref.unsafe_lo <= ref.unsafe_hi <= r["unsafe_hi"]
    assert r["boxes"] >= ref.boxes


def test_bounded_wait_gives_up_and_context_survives(pkg):
    """Failure detection: the tensor-core kernels' bounded wait, on a barrier
    nothing completes, returns SLR_ETIMEOUT; the context then counts correctly."""
    p = gen.make("tiny")
    with _counter(pkg, p) as c:
        with pytest.raises(pkg.SlrError, match="ETIMEOUT"):
            c.wait_selfcheck(4096)
        with pytest.raises(pkg.SlrError, match="EINVAL"):
            c.wait_selfcheck(0)
        r = c.count(10)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, 10)
    assert (r["unsafe_lo"], r["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
