"""The sampling-limitation experiment of Sec. 4.1 on a seeded network of its
shape (3 -> 32 -> 32 -> 1 on [0,1]^3, Q: y >= 0): the exact counter brackets a
violation rate that uniform sampling barely sees (needs a GB300)."""
import numpy as np
import pytest

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def test_rare_violation_bracket(pkg):
    p = gen.rare_violation(0)
    c = pkg.Counter(0)
    c.set_problem(p)
    # parity with the oracle at a depth it finishes quickly
    r12 = c.count(12)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, 12)
    assert (r12["unsafe_lo"], r12["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
    # deeper: a sound bracket of the tiny violation rate
    D = 24
    r = c.count(D)
    c.close()
    lo, hi = r["unsafe_lo"] / 2.0 ** D, r["unsafe_hi"] / 2.0 ** D
    assert 0 <= lo <= hi < 2e-2
    # 10^6 uniform samples: the fraction lies in the bracket up to sampling error
    rng = np.random.default_rng(7)
    x = p.lo + (p.hi - p.lo) * rng.random((1_000_000, 3))
    y = oracle.forward_points(p.net, x, p.prop)[0][:, 0]
    mc = float(np.mean(y > 0))
    sd = np.sqrt(max(hi, 1e-6) / 1e6)
    assert lo - 5 * sd <= mc <= hi + 5 * sd
    # the counter proves a positive unsafe volume: a point at a deep UNSAFE leaf is unsafe
    assert r["unsafe_hi"] > 0
