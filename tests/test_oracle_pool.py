"""The oracle's count over a process pool equals its single-process count
(CPU): same per-level statistics, bracket and leaf set; a time budget stops it
at a level boundary with the levels done so far."""
import numpy as np

import oracle
from oracle import pool
from workloads import generators as gen


def _leaf_set(codes, depth, cls):
    return sorted(zip(np.asarray(codes).tolist(), np.asarray(depth).tolist(), np.asarray(cls).tolist()))


def test_pool_count_equals_count():
    for p, D in ((gen.tiny(0), 12), (gen.acas_shaped(0), 8)):
        want = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True)
        got = pool.count_levels(p, D, procs=2, leaves=True)
        assert got["complete"]
        assert (got["unsafe_lo"], got["unsafe_hi"]) == (want.unsafe_lo, want.unsafe_hi)
        assert got["levels"] == want.levels[:len(got["levels"])]
        assert got["boxes"] == want.boxes
        w = sorted((c, t, k) for c, t, k in want.leaves)
        assert _leaf_set(got["leaf_codes"], got["leaf_depth"], got["leaf_cls"]) == w


def test_pool_budget_stops_at_a_level_boundary():
    p = gen.acas_shaped(0)
    got = pool.count_levels(p, 20, procs=2, budget_s=0.0)
    assert not got["complete"] and len(got["levels"]) == 1 and got["levels"][0]["boxes"] == 1


def test_sampled_finite_differences_equal_the_full_ones():
    """fd_gradients at chosen coordinates, in one process or dealt over a
    pool, equals the full central differences at those coordinates."""
    p = gen.tiny(0)
    rng = np.random.default_rng(2)
    lo = np.array([-0.6, -0.2])
    hi = np.array([0.1, 0.5])
    R = p.prop.C.shape[0]
    w_hi, w_lo = rng.normal(size=R), rng.normal(size=R)
    alpha = [rng.uniform(0.1, 0.9, size=w.shape[0]) for w in p.net.W[:-1]]
    full = oracle.fd_gradients(p.net, lo, hi, p.prop, alpha, w_hi, w_lo)
    a_full = np.concatenate(full["alpha"])
    a_idx, b_idx = [0, 3, 9, 14], [1]
    one = oracle.fd_gradients(p.net, lo, hi, p.prop, alpha, w_hi, w_lo, w_idx={}, alpha_idx=a_idx, box_idx=b_idx)
    many = pool.fd_gradients_sampled(p.net, lo, hi, p.prop, alpha, w_hi, w_lo, a_idx, b_idx, procs=2)
    for got_a, got_lo, got_hi in ((np.concatenate(one["alpha"]), one["lo"], one["hi"]),
                                  (many["alpha"], many["lo"], many["hi"])):
        np.testing.assert_array_equal(got_a[a_idx], a_full[a_idx])
        assert np.all(np.isnan(np.delete(got_a, a_idx)))
        np.testing.assert_array_equal(got_lo[b_idx], full["lo"][b_idx])
        np.testing.assert_array_equal(got_hi[b_idx], full["hi"][b_idx])
        assert np.isnan(got_lo[0]) and np.isnan(got_hi[0])
