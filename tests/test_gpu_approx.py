"""The approximate counter CountingProVe_SLR (Sec. 2.3; Table 1) through the C
ABI against the oracle's restatement (needs a GB300): the same draws give the
same split points, coins, leaf boxes (bit for bit), leaf counts and
estimates; without splits it is slr_count; the reported lower bound lies
below the exact count's upper end."""
import numpy as np
import pytest

from oracle import approx
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _both(pkg, p, **kw):
    with pkg.Counter(0) as c:
        c.set_problem(p)
        got = c.count_approx(**kw)
    want = approx.count_approx(p.net, p.lo, p.hi, p.prop, **kw)
    return got, want


@pytest.mark.parametrize("name,kw", [
    ("tiny", dict(trials=4, splits=6, samples=1024, leaf_depth=10, beta=1.0, seed=1)),
    ("acas", dict(trials=4, splits=8, samples=2048, leaf_depth=10, beta=1.0, seed=2)),
    ("acas", dict(trials=3, splits=12, samples=333, leaf_depth=6, beta=0.5, seed=77)),
    ("nav", dict(trials=2, splits=10, samples=4096, leaf_depth=8, beta=2.0, seed=3)),
])
def test_approx_matches_oracle(pkg, name, kw):
    p = gen.make(name)
    got, want = _both(pkg, p, **kw)
    assert got["trials"] == kw["trials"]
    for t, w in enumerate(want.trials):
        assert got["splits_done"][t] == w.splits, t
        assert np.array_equal(got["leaf_lo"][t], w.leaf_lo) and np.array_equal(got["leaf_hi"][t], w.leaf_hi), t
        assert (got["leaf_unsafe_lo"][t], got["leaf_unsafe_hi"][t]) == (w.unsafe_lo, w.unsafe_hi), t
        assert got["leaf_volume"][t] == w.volume and got["estimate"][t] == w.estimate, t
        assert got["estimate_hi"][t] == w.estimate_hi, t
    assert got["samples_unsafe"] == sum(w.samples_unsafe for w in want.trials)
    assert got["vr_lower"] == want.vr_lower and got["vr_mean"] == want.vr_mean
    assert got["confidence"] == want.confidence


def test_without_splits_it_is_the_exact_count(pkg):
    p = gen.make("acas")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        r = c.count(12)
        a = c.count_approx(trials=2, splits=0, leaf_depth=12, beta=1.0)
        again = c.count(12)                       # the context's own box is back
    assert a["splits_done"] == [0, 0]
    assert a["leaf_unsafe_lo"] == [r["unsafe_lo"]] * 2 and a["leaf_unsafe_hi"] == [r["unsafe_hi"]] * 2
    assert a["estimate"][0] == r["unsafe_lo"] / 2 ** 12
    assert (again["unsafe_lo"], again["unsafe_hi"]) == (r["unsafe_lo"], r["unsafe_hi"])


def test_lower_bound_below_the_exact_bracket(pkg):
    """ACAS-shaped: the lower bound (confidence 1 - 2^-8) lies below the exact
    count's upper end at depth 20, and the mean estimate inside a wide band."""
    p = gen.make("acas")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        exact = c.count(20)
        a = c.count_approx(trials=8, splits=10, samples=4096, leaf_depth=10, beta=1.0, seed=5)
    hi = exact["unsafe_hi"] / 2 ** 20
    lo = exact["unsafe_lo"] / 2 ** 20
    assert a["confidence"] == 1 - 2 ** -8
    assert 0.0 <= a["vr_lower"] <= hi
    assert a["vr_mean"] <= 64 * hi and a["samples_unsafe"] > 0
    assert lo <= hi


def test_approx_option_errors(pkg):
    p = gen.make("tiny")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        for bad in (dict(trials=0), dict(trials=65), dict(splits=-1), dict(samples=0), dict(samples=1 << 24),
                    dict(leaf_depth=63), dict(beta=0.0), dict(beta=float("nan"))):
            with pytest.raises(pkg.SlrError) as ei:
                c.count_approx(**bad)
            assert ei.value.code == -1, bad
