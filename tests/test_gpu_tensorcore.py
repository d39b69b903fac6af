"""Tensor-core (tcgen05, split TF32) evaluation against the FP64 oracle (needs a GB300)."""
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
    c.set_options(precision=pkg.PREC_TC_TF32, **opt)
    return c


@pytest.mark.parametrize("name", ["tiny", "acas", "nav"])
@pytest.mark.parametrize("n", [1, 37, 1000])
@pytest.mark.parametrize("shrink", [1, 16])
def test_tc_bounds_match_oracle(pkg, name, n, shrink):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, n, seed=n + shrink)
    hi = (lo + (hi - lo) / shrink).astype(np.float32)
    with _counter(pkg, p) as c:
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    # sound: the widened bounds contain the oracle's
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    raw_lo = rl.astype(np.float64) + err
    raw_hi = rh.astype(np.float64) - err
    elo, ehi, _ = bound_errors(raw_lo, raw_hi, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL, (elo.max(), ehi.max())
    dec = cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], oracle.classify(olo, ohi, p.prop)[dec])


@pytest.mark.parametrize("name,D", [("tiny", 16), ("acas", 11), ("nav", 9)])
def test_tc_count_matches_oracle(pkg, name, D):
    p = gen.make(name)
    with _counter(pkg, p, record_leaves=1) as c:
        got = c.count(D)
        codes, depth, cls = c.leaves()
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True)
    assert (got["unsafe_lo"], got["unsafe_hi"]) == (want.unsafe_lo, want.unsafe_hi)
    assert got["level_boxes"] == [lv["boxes"] for lv in want.levels]
    assert sorted(zip(codes.tolist(), depth.tolist(), cls.tolist())) == sorted(want.leaves)


def test_tc_full_depth_equals_fp32_path(pkg):
    p = gen.acas_shaped(0)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        ref = c.count(p.depth)
        c.set_options(precision=pkg.PREC_TC_TF32)
        got = c.count(p.depth)
    for k in ("unsafe_lo", "unsafe_hi", "boxes", "level_boxes", "level_safe", "level_unsafe", "level_undecided"):
        assert got[k] == ref[k], k


def test_tc_sound_on_a_million_points(pkg):
    p = gen.nav_shaped(0)
    lo, hi = random_sub_boxes(p, 16, seed=4)
    lo[0], hi[0] = p.lo, p.hi
    with _counter(pkg, p) as c:
        rl, rh, _ = c.bounds(lo, hi)
    rng = np.random.default_rng(12)
    for k in range(16):
        x = lo[k].astype(np.float64) + (hi[k].astype(np.float64) - lo[k]) * rng.random((62500, p.d))
        rows, _ = oracle.forward_points(p.net, x, p.prop)
        assert np.all(rows >= rl[k]) and np.all(rows <= rh[k]), k


def test_tc_rejects_wide_networks(pkg):
    rng = np.random.default_rng(0)
    net = gen._mlp(rng, [4, 96, 3])
    p = gen.Problem("wide", net, np.zeros(4, np.float32), np.ones(4, np.float32), gen.tiny(0).prop, 6, 0)
    p.prop = gen._prop([[(gen._unit(3, 0), 0.0, False)]])
    c = pkg.Counter(0)
    c.set_problem(p)
    c.set_options(precision=pkg.PREC_TC_TF32)
    with pytest.raises(pkg.SlrError) as ei:
        c.count(4)
    assert ei.value.code == -7
    c.close()
