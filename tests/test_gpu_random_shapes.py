"""Randomised parity over network and property shapes (needs a GB300): each
case draws a small ReLU network (1-4 affine layers, widths 1-40, 1-9 inputs),
an input box (some dimensions of zero width), and a property of 1-3 clauses
of 1-3 strict or non-strict rows; counts must equal the oracle's bit for bit
(FP32 tile path, tensor-core tile path where the widths allow, wide path
equal, its FP64 re-check included), and bounds must agree within the bar."""
import numpy as np
import pytest

import oracle
from workloads.generators import Network, Problem, Property

from .gpu_common import BOUND_RTOL, bound_errors, random_sub_boxes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    K = int(rng.integers(1, 5))
    d = int(rng.integers(1, 10))
    widths = [d] + [int(rng.integers(1, 41)) for _ in range(K - 1)] + [int(rng.integers(1, 5))]
    W, b = [], []
    for k in range(K):
        W.append(rng.normal(0, np.sqrt(2.0 / widths[k]), size=(widths[k + 1], widths[k])).astype(np.float32))
        b.append(rng.normal(0, 0.3, size=widths[k + 1]).astype(np.float32))
    centre = rng.uniform(-1, 1, size=d)
    half = rng.uniform(0.05, 0.8, size=d)
    half[rng.random(d) < 0.2] = 0.0                       # zero-width dimensions
    lo = (centre - half).astype(np.float32)
    hi = (centre + half).astype(np.float32)
    n_out = widths[-1]
    clauses, rows = int(rng.integers(1, 4)), []
    rpc = []
    for _ in range(clauses):
        nr = int(rng.integers(1, 4))
        rpc.append(nr)
        for _ in range(nr):
            rows.append((rng.normal(size=n_out).astype(np.float32), np.float32(rng.normal(0, 0.3)),
                         int(rng.random() < 0.5)))
    prop = Property(rows_per_clause=np.array(rpc, np.int32), C=np.array([r[0] for r in rows], np.float32),
                    e=np.array([r[1] for r in rows], np.float32), strict=np.array([r[2] for r in rows], np.uint8))
    return Problem(f"random_{seed}", Network(W, b), lo, hi, prop, 10, seed)


@pytest.mark.parametrize("seed", range(24))
def test_random_shape_counts(pkg, seed):
    p = _case(seed)
    D = p.depth
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D)
    c = pkg.Counter(0)
    c.set_problem(p)
    r = c.count(D)
    assert (r["unsafe_lo"], r["unsafe_hi"], r["boxes"]) == (ref.unsafe_lo, ref.unsafe_hi, ref.boxes)
    # bounds of random sub-boxes
    lo, hi = random_sub_boxes(p, 64, seed=seed)
    rl, rh, cls, err = c.bounds(lo, hi, want_err=True)
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL
    # the wide path gives the same count (its NEAR boxes re-bounded in FP64)
    c.set_options(wide=1)
    w = c.count(D)
    assert w["tie_leaves"] == 0
    assert (w["unsafe_lo"], w["unsafe_hi"], w["boxes"]) == (ref.unsafe_lo, ref.unsafe_hi, ref.boxes)
    # the tensor-core tile path where it applies (a hidden layer, widths <= 64)
    if p.net.K >= 2:
        c.set_options(precision=pkg.PREC_TC_TF32)
        t = c.count(D)
        assert (t["unsafe_lo"], t["unsafe_hi"], t["boxes"]) == (ref.unsafe_lo, ref.unsafe_hi, ref.boxes)
    c.close()
