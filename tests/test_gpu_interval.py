"""Interval mode (Moore intervals, the paper's naive Exact Count baseline of
Sec. 4) against the oracle's interval count, through the C ABI (needs a GB300)."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen

from .gpu_common import random_sub_boxes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


@pytest.mark.parametrize("name,D", [("tiny", 14), ("acas", 13), ("nav", 12)])
@pytest.mark.parametrize("wide", [0, 1])
def test_interval_count_matches_oracle(pkg, name, D, wide):
    p = gen.make(name)
    c = pkg.Counter(0)
    c.set_problem(p)
    c.set_options(relax_mode=pkg.RELAX_INTERVAL, wide=wide)
    r = c.count(D)
    c.close()
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D, bound="interval")
    if wide and r["tie_leaves"]:
        assert r["unsafe_lo"] <= ref.unsafe_lo <= ref.unsafe_hi <= r["unsafe_hi"]
    else:
        assert (r["unsafe_lo"], r["unsafe_hi"], r["boxes"]) == (ref.unsafe_lo, ref.unsafe_hi, ref.boxes)


def test_interval_bounds_match_oracle(pkg):
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 300, seed=3)
    c = pkg.Counter(0)
    c.set_problem(p)
    c.set_options(relax_mode=pkg.RELAX_INTERVAL)
    rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    c.close()
    olo, ohi = oracle.interval_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)[:2]
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    assert np.max(np.abs(rl + err - olo) / scale) <= 1e-5 and np.max(np.abs(rh - err - ohi) / scale) <= 1e-5
