"""The synthetic inputs against their stated recipe (CPU).

Every parity case and the benchmark run on these seeded stand-ins for the
paper's networks, so their recipe is pinned here: shapes and dtypes, He
weights N(0, 2/fan_in) and biases N(0, 0.1), the boxes, the unsafe sets, the
violation-rate windows the seeds were chosen for, and bit-identical
regeneration from a seed.  The forward pass and the property test below are
written out here in float64; the generators' own seed-selection pass is not
reused."""
import numpy as np
import pytest

from workloads import generators as gen

MC_SAMPLES = 1 << 16


def _forward64(net, x):
    h = np.asarray(x, np.float64)
    for k in range(net.K):
        h = h @ np.asarray(net.W[k], np.float64).T + np.asarray(net.b[k], np.float64)
        if k < net.K - 1:
            h = np.maximum(h, 0.0)
    return h


def _unsafe64(prop, y):
    vals = y @ np.asarray(prop.C, np.float64).T + np.asarray(prop.e, np.float64)
    sat = np.where(prop.strict.astype(bool), vals > 0, vals >= 0)
    out = np.zeros(y.shape[0], bool)
    r = 0
    for nr in prop.rows_per_clause:
        out |= sat[:, r:r + int(nr)].all(axis=1)
        r += int(nr)
    return out


def _rate(p, n=MC_SAMPLES, seed=2024):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(p.lo, np.float64), np.asarray(p.hi, np.float64)
    x = lo + (hi - lo) * rng.random((n, p.d))
    return float(_unsafe64(p.prop, _forward64(p.net, x)).mean())


def _within(rate, window, n=MC_SAMPLES):
    """The window widened by five standard errors of an n-sample estimate."""
    lo, hi = window
    sd = np.sqrt(max(rate * (1 - rate), 1.0 / n) / n)
    return lo - 5 * sd <= rate <= hi + 5 * sd


SHAPES = {
    "tiny": [2, 8, 8, 1],
    "acas": [5] + [50] * 6 + [5],
    "nav": [22, 64, 64, 3],
    "mnist": [784, 256, 256, 256, 10],
    "rare": [3, 32, 32, 1],
}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_shapes_dtypes_and_regeneration(name):
    p = gen.make(name)
    assert p.net.widths == SHAPES[name]
    for W, b in zip(p.net.W, p.net.b):
        assert W.dtype == np.float32 and b.dtype == np.float32
    assert p.lo.dtype == np.float32 and p.hi.dtype == np.float32 and np.all(p.lo < p.hi)
    assert p.prop.C.shape == (p.prop.R, SHAPES[name][-1]) and p.prop.C.dtype == np.float32
    assert int(p.prop.rows_per_clause.sum()) == p.prop.R
    fresh = getattr(gen.CONFIGS[name], "__wrapped__", gen.CONFIGS[name])(0)     # past the generator's cache
    for a, b in zip(p.net.W + p.net.b + [p.lo, p.hi, p.prop.C, p.prop.e],
                    fresh.net.W + fresh.net.b + [fresh.lo, fresh.hi, fresh.prop.C, fresh.prop.e]):
        assert a.tobytes() == b.tobytes()


@pytest.mark.parametrize("name", ["acas", "nav", "mnist"])
def test_he_weights_and_bias_variance(name):
    p = gen.make(name)
    for W in p.net.W:
        if W.size < 1000:
            continue
        fan_in = W.shape[1]
        assert abs(float(W.mean())) < 4 * np.sqrt(2.0 / fan_in / W.size)
        assert abs(float(W.var()) / (2.0 / fan_in) - 1.0) < 0.15
    b = np.concatenate(p.net.b)
    assert abs(float(b.var()) / 0.1 - 1.0) < 0.35


def test_boxes_follow_their_recipes():
    eps = 1e-6
    t = gen.make("tiny")
    assert np.all(t.lo == -1) and np.all(t.hi == 1)
    a = gen.make("acas")
    side = a.hi.astype(np.float64) - a.lo
    assert np.all(side >= 0.05 - eps) and np.all(side <= 0.3 + eps)
    assert np.all(a.lo >= -0.5 - eps) and np.all(a.hi <= 0.5 + eps)
    n = gen.make("nav")
    w = n.hi.astype(np.float64) - n.lo
    c = (n.hi.astype(np.float64) + n.lo) / 2
    assert np.allclose(w[:20], 0.05, atol=eps) and np.allclose(w[20:], 0.01, atol=eps)
    assert np.all((c[:20] >= 0.025 - eps) & (c[:20] <= 0.975 + eps))
    assert np.all((c[20:] >= -0.995 - eps) & (c[20:] <= 0.995 + eps))
    m = gen.make("mnist")
    x0 = m.extra["centre"].astype(np.float64)
    assert np.allclose(m.lo, np.clip(x0 - 0.02, 0, 1), atol=eps)
    assert np.allclose(m.hi, np.clip(x0 + 0.02, 0, 1), atol=eps)
    r = gen.make("rare")
    assert np.all(r.lo == 0) and np.all(r.hi == 1)


def test_unsafe_sets_follow_their_recipes():
    a = gen.make("acas").prop          # OR_j y_0 - y_j > 0
    assert list(a.rows_per_clause) == [1, 1, 1, 1] and np.all(a.strict == 1) and np.all(a.e == 0)
    for j in range(1, 5):
        want = np.zeros(5, np.float32)
        want[0], want[j] = 1, -1
        assert np.array_equal(a.C[j - 1], want)
    n = gen.make("nav").prop           # y_1 >= y_0 and y_1 >= y_2
    assert list(n.rows_per_clause) == [2] and np.all(n.strict == 0)
    assert np.array_equal(n.C, np.array([[-1, 1, 0], [0, 1, -1]], np.float32))
    m = gen.make("mnist").prop         # OR_{j>0} y_j - y_0 >= 0
    assert list(m.rows_per_clause) == [1] * 9 and np.all(m.strict == 0)
    assert np.all(m.C[:, 0] == -1) and np.array_equal(m.C[:, 1:], np.eye(9, dtype=np.float32))
    for name in ("tiny", "rare"):      # y < 0
        q = gen.make(name).prop
        assert q.R == 1 and q.strict[0] == 1 and q.C[0, 0] == -1 and q.e[0] == 0


@pytest.mark.parametrize("name,window", [("tiny", (0.05, 0.95)), ("acas", (0.005, 0.5)), ("nav", (0.05, 0.5))])
def test_violation_rate_lies_in_the_selection_window(name, window):
    assert _within(_rate(gen.make(name)), window)


def test_mnist_centre_is_class_zero():
    m = gen.make("mnist")
    y = _forward64(m.net, m.extra["centre"][None])[0]
    assert int(np.argmax(y)) == 0


def test_rare_violation_grid_minimum_and_rate():
    r = gen.make("rare")
    g = np.linspace(0.0, 1.0, 65)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ymin = float(_forward64(r.net, grid).min())
    assert abs(ymin - (-2e-3)) < 1e-5
    assert _rate(r) < 0.01


def test_batched_members_follow_their_recipe():
    probs = gen.batched_uneven(1, n_nets=4, props_per_net=3, depth_range=(6, 11))
    assert len(probs) == 12
    for p in probs:
        w = p.net.widths
        d, hidden = w[0], w[1:-1]
        assert d in (5, 8, 16, 32)
        assert len(set(hidden)) == 1 and hidden[0] in (32, 64, 128) and 2 <= len(hidden) <= 8
        assert (2 * d + 3) * ((hidden[0] + 7) // 8) <= 512        # kept only where the tile holds it
        assert 2 <= w[-1] <= 8 and 6 <= p.depth <= 11
        side = p.hi.astype(np.float64) - p.lo
        assert np.all(side >= 0.02 - 1e-6) and np.all(side <= 0.2 + 1e-6)
        assert np.all(p.lo >= -0.5 - 1e-6) and np.all(p.hi <= 0.5 + 1e-6)
        assert len(p.prop.rows_per_clause) == 1
        assert 1 <= p.prop.R <= 2 and np.all(p.prop.strict == 0)
        for row in p.prop.C:
            nz = np.nonzero(row)[0]
            assert len(nz) == 2 and row[nz].max() > 0 > row[nz].min()
            assert np.all((np.abs(row[nz]) >= 0.5 - 1e-6) & (np.abs(row[nz]) <= 2.0 + 1e-6))
        assert _within(_rate(p, n=1 << 14), (0.01, 0.99), n=1 << 12)
