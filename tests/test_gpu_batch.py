"""Batched counting of many uneven problems in one persistent launch per step (needs a GB300)."""
import copy

import numpy as np
import pytest

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu

KEYS = ("unsafe_lo", "unsafe_hi", "boxes", "level_boxes", "level_safe", "level_unsafe", "level_undecided")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _mixed():
    probs = [gen.tiny(0), gen.tiny(1), gen.tiny(2), gen.acas_shaped(0), gen.nav_shaped(0), gen.rare_violation(0),
             gen.linear_2d(1, 10), gen.single_layer_1d(3, depth=12)]
    depths = [16, 12, 9, 10, 8, 12, 10, 12]
    probs += gen.batched_uneven(1, n_nets=4, props_per_net=3, depth_range=(6, 11))
    depths += [p.depth for p in probs[8:]]
    return probs, depths


def _single(pkg, p, D):
    with pkg.Counter(0) as c:
        c.set_problem(p)
        return c.count(D)


def test_batch_equals_single_counts(pkg):
    probs, depths = _mixed()
    with pkg.Counter(0) as c:
        got = c.count_batch(probs, depths)
        again = c.count_batch(probs, depths)          # replayed graph, counters cleared
    for p, D, g, a in zip(probs, depths, got, again):
        want = _single(pkg, p, D)
        for k in KEYS:
            assert g[k] == want[k], (p.name, D, k)
            assert a[k] == want[k], (p.name, D, k, "replay")


def test_batch_matches_oracle_on_small_problems(pkg):
    probs = [gen.tiny(0), gen.tiny(3), gen.linear_2d(2, 10), gen.acas_shaped(1)]
    depths = [14, 12, 10, 9]
    with pkg.Counter(0) as c:
        got = c.count_batch(probs, depths)
    for p, D, g in zip(probs, depths, got):
        s = _single(pkg, p, D)
        for k in KEYS:
            assert np.array_equal(np.asarray(g[k]), np.asarray(s[k])), (p.name, k)
        w = oracle.count(p.net, p.lo, p.hi, p.prop, D)
        assert (g["unsafe_lo"], g["unsafe_hi"]) == (w.unsafe_lo, w.unsafe_hi), p.name
        assert g["level_boxes"] == [lv["boxes"] for lv in w.levels]


def test_batch_new_weights_same_shape(pkg):
    """A second call with the same shapes reuses the captured graph with the new data."""
    probs, depths = _mixed()
    with pkg.Counter(0) as c:
        c.count_batch(probs, depths)
        moved = []
        for i, p in enumerate(probs):
            q = copy.deepcopy(p)
            rng = np.random.default_rng(100 + i)
            q.net.b[0] = (q.net.b[0] + rng.normal(0, 0.05, size=q.net.b[0].shape)).astype(np.float32)
            moved.append(q)
        got = c.count_batch(moved, depths)
    for q, D, g in zip(moved, depths, got):
        want = _single(pkg, q, D)
        assert all(g[k] == want[k] for k in KEYS), q.name


def test_batch_rejects_bad_problem(pkg):
    p = copy.deepcopy(gen.tiny(0))
    p.lo = np.array([1.0, 0.0], np.float32)
    p.hi = np.array([0.0, 1.0], np.float32)
    with pkg.Counter(0) as c:
        with pytest.raises(pkg.SlrError) as ei:
            c.count_batch([gen.tiny(1), p], [8, 8])
        assert ei.value.code == -1 and "problem 1" in str(ei.value)


def test_batch_with_wide_members(pkg):
    """256- and 512-wide members run on the wide path inside the same batched call."""
    probs = [gen.tiny(0), gen.acas_shaped(0)]
    depths = [12, 9]
    probs += gen.batched_uneven(4, n_nets=2, props_per_net=2, depth_range=(6, 8), widths=(256, 512), tile_only=False)
    depths += [p.depth for p in probs[2:]]
    assert any(max(p.net.widths[1:-1]) >= 256 for p in probs)
    with pkg.Counter(0) as c:
        got = c.count_batch(probs, depths)
    for p, D, g in zip(probs, depths, got):
        s = _single(pkg, p, D)
        for k in KEYS:
            assert np.array_equal(np.asarray(g[k]), np.asarray(s[k])), (p.name, k)
        w = oracle.count(p.net, p.lo, p.hi, p.prop, D)
        if g["tie_leaves"] == 0:
            assert (g["unsafe_lo"], g["unsafe_hi"]) == (w.unsafe_lo, w.unsafe_hi), p.name
        else:
            assert g["unsafe_lo"] <= w.unsafe_lo <= w.unsafe_hi <= g["unsafe_hi"], p.name


def test_batch_rechecks_beside_wide_members(pkg):
    """A problem whose every level needs the FP64 re-check, batched with the
    widest members of the mixed batch: the batch's FP64 tile must hold the
    largest shape, and the re-checked problem still equals its single count."""
    from .test_gpu_parity import _margin_at_a_corner
    corner = _margin_at_a_corner()
    probs, depths = _mixed()
    probs, depths = [corner] + probs[8:], [corner.depth] + depths[8:]
    with pkg.Counter(0) as c:
        got = c.count_batch(probs, depths)
    assert got[0]["rechecked"] > 0 and got[0]["tie_leaves"] == 0
    want = _single(pkg, corner, corner.depth)
    for k in KEYS:
        assert got[0][k] == want[k], k
