"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen

from .gpu_common import BOUND_RTOL, bound_errors, leaves_partition_root, oracle_classes_of, random_sub_boxes

pytestmark = pytest.mark.gpu

CONFIGS = ["tiny", "acas", "nav"]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _counter(pkg, p, **opt):
    c = pkg.Counter(0)
    c.set_problem(p)
    if opt:
        c.set_options(**opt)
    return c


# ---------------------------------------------------------------------------
# bounds
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", CONFIGS)
@pytest.mark.parametrize("n", [1, 7, 133, 1000])
def test_bounds_match_oracle(pkg, name, n):
    """Row bounds of random sub-boxes (several tiles plus a ragged tail) agree with the oracle."""
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, n, seed=n)
    with _counter(pkg, p) as c:
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    # the widened bounds contain the oracle's (rounding of the FP64 oracle aside)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale), "GPU lower bound above the exact SLR bound"
    assert np.all(rh >= ohi - 1e-12 * scale), "GPU upper bound below the exact SLR bound"
    # the FP32 SLR bounds themselves (widening removed) agree within BOUND_RTOL
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL, (elo.max(), ehi.max())
    ocls = oracle.classify(olo, ohi, p.prop)
    # a GPU decision is always the oracle's decision; undecided may differ only within rounding
    dec = cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], ocls[dec])


@pytest.mark.parametrize("name", CONFIGS)
def test_bounds_are_sound_on_a_million_points(pkg, name):
    """10^6 sampled points per configuration fall inside the GPU row bounds."""
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, 16, seed=3)
    lo[0], hi[0] = p.lo, p.hi
    with _counter(pkg, p) as c:
        rl, rh, _ = c.bounds(lo, hi)
    rng = np.random.default_rng(11)
    per = 1_000_000 // 16
    for k in range(16):
        x = lo[k].astype(np.float64) + (hi[k].astype(np.float64) - lo[k]) * rng.random((per, p.d))
        rows, _ = oracle.forward_points(p.net, x, p.prop)
        assert np.all(rows >= rl[k]) and np.all(rows <= rh[k]), k


def test_bounds_device_pointers_match_host(pkg):
    torch = pytest.importorskip("torch")
    p = gen.acas_shaped(0)
    lo, hi = random_sub_boxes(p, 300, seed=5)
    with _counter(pkg, p) as c:
        rl, rh, cls = c.bounds(lo, hi)
        tl, th, tc = c.bounds(torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda())
    assert np.array_equal(rl, tl.cpu().numpy()) and np.array_equal(rh, th.cpu().numpy())
    assert np.array_equal(cls, tc.cpu().numpy())


def test_degenerate_boxes(pkg):
    """Zero-width sides and point boxes: bounds collapse onto the network value."""
    p = gen.acas_shaped(0)
    lo, hi = random_sub_boxes(p, 40, seed=9)
    hi[:20, 2] = lo[:20, 2]
    hi[20:] = lo[20:]
    with _counter(pkg, p) as c:
        rl, rh, _, err = c.bounds(lo, hi, want_err=True)
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL
    rows, _ = oracle.forward_points(p.net, lo[20:].astype(np.float64), p.prop)
    assert np.all(rl[20:] <= rows) and np.all(rows <= rh[20:])


# ---------------------------------------------------------------------------
# counts
# ---------------------------------------------------------------------------

def _check_count(pkg, p, D, **opt):
    with _counter(pkg, p, record_leaves=1, **opt) as c:
        got = c.count(D)
        codes, depth, cls = c.leaves()
        sched = c.schedule(D)
    want = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True,
                        mode="paper_literal" if opt.get("relax_mode") == 1 else "neurify")
    assert np.array_equal(sched, oracle.split_schedule(p.lo, p.hi, D))
    assert (got["unsafe_lo"], got["unsafe_hi"]) == (want.unsafe_lo, want.unsafe_hi), (got, want.unsafe_lo, want.unsafe_hi)
    for t, lv in enumerate(want.levels):
        assert got["level_boxes"][t] == lv["boxes"]
        assert got["level_safe"][t] == lv["safe"]
        assert got["level_unsafe"][t] == lv["unsafe"]
        assert got["level_undecided"][t] == lv["undecided"]
    g = sorted(zip(codes.tolist(), depth.tolist(), cls.tolist()))
    w = sorted((c_, t_, k_) for c_, t_, k_ in want.leaves)
    assert g == w
    return got


@pytest.mark.parametrize("name,D", [("tiny", 16), ("acas", 11), ("nav", 9)])
def test_count_matches_oracle(pkg, name, D):
    got = _check_count(pkg, gen.make(name), D)
    assert got["tie_leaves"] == 0


def test_count_paper_literal_reading(pkg):
    _check_count(pkg, gen.tiny(0), 14, relax_mode=1)


@pytest.mark.parametrize("D", [0, 1, 2])
def test_shallow_counts(pkg, D):
    _check_count(pkg, gen.acas_shaped(0), D)


def test_linear_network_count(pkg):
    """One affine layer (no ReLU): counts equal the oracle's."""
    _check_count(pkg, gen.linear_2d(3, 12), 12)


def test_one_dimensional_network(pkg):
    _check_count(pkg, gen.single_layer_1d(2, depth=14), 14)


def test_other_seeds_match(pkg):
    for s in (1, 2):
        _check_count(pkg, gen.tiny(s), 16)
        _check_count(pkg, gen.acas_shaped(s), 10)


def test_full_depth_acas_sampled_leaves(pkg):
    """Depth 20 on the ACAS-shaped net: leaves tile the root and sampled leaves match the oracle."""
    p = gen.acas_shaped(0)
    D = p.depth
    with _counter(pkg, p, record_leaves=1) as c:
        got = c.count(D)
        codes, depth, cls = c.leaves()
    assert leaves_partition_root(codes, depth, D)
    lo = sum(1 << (D - int(t)) for t, k in zip(depth, cls) if k == oracle.UNSAFE)
    und = int(np.count_nonzero((cls == oracle.UNDECIDED) & (depth == D)))
    assert (lo, lo + und) == (got["unsafe_lo"], got["unsafe_hi"])
    rng = np.random.default_rng(1)
    sel = rng.choice(len(codes), size=min(3000, len(codes)), replace=False)
    ocls = oracle_classes_of(p, codes[sel].astype(np.int64), depth[sel], D)
    assert np.array_equal(ocls, cls[sel].astype(np.int8))
    # every ancestor of a sampled leaf was undecided in the oracle too
    anc_codes, anc_depth = [], []
    for cd, t in zip(codes[sel[:300]].tolist(), depth[sel[:300]].tolist()):
        for s in range(t):
            anc_codes.append(cd >> (t - s))
            anc_depth.append(s)
    acls = oracle_classes_of(p, np.array(anc_codes, dtype=np.int64), np.array(anc_depth), D)
    assert np.all(acls == oracle.UNDECIDED)


def test_determinism(pkg):
    p = gen.acas_shaped(0)
    with _counter(pkg, p, record_leaves=1) as c:
        a = c.count(14)
        la = sorted(zip(*[x.tolist() for x in c.leaves()]))
        b = c.count(14)
        lb = sorted(zip(*[x.tolist() for x in c.leaves()]))
    for k in ("device_ms", "kernel_ms", "h2d_bytes", "d2h_bytes"):   # timings and copies, not results
        a.pop(k)
        b.pop(k)
    assert a == b and la == lb


def _recheck_both_ways(pkg, p, D):
    """Both re-check forms on the same FP32 tile (the autotuner of two contexts
    may time two tiles differently, and the tile fixes which boxes are NEAR)."""
    out = []
    tile = {}
    for cl in (1, 0):
        with _counter(pkg, p, record_leaves=1, recheck_cluster=cl, **tile) as c:
            r = c.count(D)
            leaves = sorted(zip(*[x.tolist() for x in c.leaves()]))
        tile = dict(tile_boxes=r["tile"][0], tile_threads=r["tile"][1])
        # the one-CTA form runs its float-float stage first: one more launch a
        # level, and fewer boxes left to plain FP64 products
        for k in ("device_ms", "kernel_ms", "h2d_bytes", "d2h_bytes", "launches", "rechecked_fp64"):
            r.pop(k)
        out.append((r, leaves))
    return out


@pytest.mark.parametrize("name,D", [("acas", 17), ("nav", 12), ("tiny", 16)])
def test_recheck_on_clusters_matches_single_cta(pkg, name, D):
    """The FP64 re-check with each tile over a cluster of CTAs gives the
    classes of the one-CTA tile (both sound; only the products' summation
    order differs).  ACAS-shaped: two-box tiles (odd input count)."""
    a, b = _recheck_both_ways(pkg, gen.make(name), D)
    if name == "acas":
        assert a[0]["rechecked"] > 0
    assert a == b


def _margin_at_a_corner(seed=0, width=32, D=12):
    """2 -> width -> width -> 1 with dyadic weights, every neuron active on
    the whole box [-1, 1]^2, so that y is linear there and y(0) = 0 exactly;
    unsafe: y - 1e-12 >= 0.  The origin is a corner of boxes at every depth:
    those on either side of the line y = 0 have a margin of -+1e-12, far
    inside the float32 widening and far outside float64's, so every level
    sends boxes to the FP64 re-check, which decides them as the oracle does."""
    rng = np.random.default_rng(seed)
    W1 = rng.integers(1, 8, size=(width, 2)) / 64.0          # pre-activation >= 1 - 14/64
    W2 = rng.integers(-8, 9, size=(width, width)) / 512.0    # |W2 h1| <= width * 8/512 * 1.22
    W3 = rng.integers(-16, 17, size=(1, width)) / 64.0
    b1 = np.ones(width)
    b2 = np.ones(width)
    h2 = W2 @ b1 + b2                                         # at x = 0, exact in float64
    b3 = -(W3 @ h2)
    net = gen.Network([w.astype(np.float32) for w in (W1, W2, W3)],
                      [v.astype(np.float32) for v in (b1, b2, b3)])
    assert float(b3[0]) == float(np.float32(b3[0]))
    prop = gen._prop([[(np.ones(1, dtype=np.float32), -1e-12, False)]])
    lo = np.full(2, -1.0, dtype=np.float32)
    hi = np.full(2, 1.0, dtype=np.float32)
    return gen.Problem("corner_margin_2-32-32-1", net, lo, hi, prop, D, seed)


def test_recheck_on_clusters_even_inputs(pkg):
    """Four-box tiles (even input count), both ways against the oracle."""
    p = _margin_at_a_corner()
    got = [_check_count(pkg, p, p.depth, recheck_cluster=cl) for cl in (1, 0)]
    assert got[0]["rechecked"] > 0 and got[0]["tie_leaves"] == 0
    assert got[0]["rechecked"] == got[1]["rechecked"]


def test_without_recheck_is_still_sound(pkg):
    """With the FP64 re-check off, the GPU bracket contains the oracle's."""
    p = gen.acas_shaped(0)
    with _counter(pkg, p, fp64_recheck=0) as c:
        got = c.count(12)
    want = oracle.count(p.net, p.lo, p.hi, p.prop, 12)
    assert got["unsafe_lo"] <= want.unsafe_lo and got["unsafe_hi"] >= want.unsafe_hi


# ---------------------------------------------------------------------------
# error paths
# ---------------------------------------------------------------------------

def test_frontier_overflow_is_reported(pkg):
    p = gen.acas_shaped(0)
    with _counter(pkg, p, frontier_cap=64) as c:
        with pytest.raises(pkg.SlrError) as ei:
            c.count(12)
        assert ei.value.code == -5


def test_call_order_and_arguments(pkg):
    p = gen.tiny(0)
    c = pkg.Counter(0)
    with pytest.raises(pkg.SlrError) as ei:
        c.count(4)
    assert ei.value.code == -4
    c.set_problem(p)
    for D in (-1, 63):
        with pytest.raises(pkg.SlrError) as ei:
            c.count(D)
        assert ei.value.code == -1
    with pytest.raises(pkg.SlrError):
        c.set_box(np.array([1.0, 0.0]), np.array([0.0, 1.0]))
    with pytest.raises(pkg.SlrError):
        c.set_box(np.array([np.nan, 0.0]), np.array([0.0, 1.0]))
    c.set_box(np.zeros(3), np.ones(3))
    with pytest.raises(pkg.SlrError) as ei:
        c.count(4)
    assert ei.value.code == -1
    c.close()


def test_replayed_level_loop_follows_changes(pkg):
    """The level loop is replayed from a captured graph: counts after a new box,
    a new property, new options and a new network equal fresh contexts' counts."""
    import copy
    p = gen.make("acas")
    q = copy.deepcopy(p)
    m = 0.5 * (p.lo.astype(np.float64) + p.hi)
    r = 0.25 * (p.hi.astype(np.float64) - p.lo)
    q.lo, q.hi = (m - r).astype(np.float32), (m + r).astype(np.float32)
    t = gen.make("acas", 10)
    D = 12

    def fresh(prob, **opt):
        with pkg.Counter(0) as c:
            c.set_problem(prob)
            if opt:
                c.set_options(**opt)
            return c.count(D)

    keys = ("unsafe_lo", "unsafe_hi", "boxes", "level_boxes", "level_undecided")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        a1 = c.count(D)
        a2 = c.count(D)
        c.set_box(q.lo, q.hi)
        b = c.count(D)
        c.set_property(t.prop.rows_per_clause, t.prop.C, t.prop.e, t.prop.strict)
        qt = copy.deepcopy(q)
        qt.prop = t.prop
        e = c.count(D)
        c.set_options(record_leaves=1)
        f = c.count(D)
        c.set_problem(t)
        g = c.count(D)
    for k in keys:
        assert a1[k] == a2[k]
    want = [(b, fresh(q)), (e, fresh(qt)), (f, fresh(qt, record_leaves=1)), (g, fresh(t))]
    for got, ref in want:
        for k in keys:
            assert got[k] == ref[k], k


def test_full_depth_acas_whole_leaf_set(pkg):
    """Depth 20 on the ACAS-shaped net, the benchmark's count: every level's
    statistics, the bracket and the whole sorted leaf set (about a million
    leaves) equal the oracle's, run level by level on a pool of host processes."""
    from oracle import pool
    p = gen.acas_shaped(0)
    D = p.depth
    with _counter(pkg, p, record_leaves=1) as c:
        got = c.count(D)
        codes, depth, cls = c.leaves()
    want = pool.count_levels(p, D, leaves=True)
    assert want["complete"]
    assert (got["unsafe_lo"], got["unsafe_hi"]) == (want["unsafe_lo"], want["unsafe_hi"])
    for t, lv in enumerate(want["levels"]):
        assert (got["level_boxes"][t], got["level_safe"][t], got["level_unsafe"][t], got["level_undecided"][t]) == \
            (lv["boxes"], lv["safe"], lv["unsafe"], lv["undecided"]), t
    assert got["tie_leaves"] == 0

    def keyed(c_, t_, k_):
        c_ = np.asarray(c_, np.int64)
        t_ = np.asarray(t_, np.int64)
        order = np.lexsort((c_, t_))
        return t_[order], c_[order], np.asarray(k_, np.int64)[order]

    gt, gc, gk = keyed(codes, depth, cls)
    wt, wc, wk = keyed(want["leaf_codes"], want["leaf_depth"], want["leaf_cls"])
    assert gt.shape == wt.shape
    assert np.array_equal(gt, wt) and np.array_equal(gc, wc) and np.array_equal(gk, wk)
