"""The gradient split rule on the GPU (a split dimension per box chosen from the
adjoint's radius gradient of the decision loss) against the FP64 oracle,
through the C ABI (needs a GB300).

The oracle replays the GPU's recorded split dimensions, so counts, levels and
leaves compare exactly; the choices themselves are checked against the
oracle's central-difference scores (near-optimal within rounding, away from
kinks)."""
import copy

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


def _shrunk(name, f):
    p = copy.deepcopy(gen.make(name))
    if f != 1.0:
        m = 0.5 * (p.lo.astype(np.float64) + p.hi)
        r = 0.5 * (p.hi.astype(np.float64) - p.lo) * f
        p.lo = (m - r).astype(np.float32)
        p.hi = (m + r).astype(np.float32)
    return p


def _gpu_count(pkg, p, D, **opt):
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(split_rule=pkg.SPLIT_GRADIENT, record_leaves=1, **opt)
        r = c.count(D)
        codes, depth, cls = c.leaves()
        S = c.split_set()
    return r, codes, depth, cls, S


def _split_map(pkg, codes, depth, S):
    """(level, path prefix) -> split dimension, from the leaves' codes; every
    leaf below a node must agree on the node's split."""
    m = {}
    for code, T in zip(codes.tolist(), depth.tolist()):
        path, dims = pkg.split_code_dims(code, T, S)
        for j in range(T):
            key = (j, path >> (T - j))
            assert m.setdefault(key, dims[j]) == dims[j]
    return m


def _replay(m):
    def choose(t, paths, lo, hi):
        return np.array([m[(t, int(q))] for q in paths], dtype=np.int64)
    return choose


def _node_box(p, path, t, m):
    """float64 endpoints of the depth-t node with the given path under the split map."""
    a = p.lo.astype(np.float64)
    w = p.hi.astype(np.float64) - a
    k = np.zeros(p.d, dtype=np.int64)
    c = np.zeros(p.d, dtype=np.int64)
    for j in range(t):
        i = m[(j, path >> (t - j))]
        k[i] = 2 * k[i] + ((path >> (t - 1 - j)) & 1)
        c[i] += 1
    s = np.ldexp(1.0, -c)
    return a + w * (k * s), a + w * ((k + 1) * s)


CASES = [("tiny", 1.0, 12), ("acas", 0.1, 12), ("nav", 0.1, 10)]


@pytest.mark.parametrize("name,f,D", CASES)
def test_gradient_count_replays_in_oracle(pkg, name, f, D):
    p = _shrunk(name, f)
    r, codes, depth, cls, S = _gpu_count(pkg, p, D)
    assert r["tie_leaves"] == 0
    m = _split_map(pkg, codes, depth, S)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D, collect_leaves=True, split=_replay(m))
    assert (r["unsafe_lo"], r["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
    assert r["level_boxes"] == [lv["boxes"] for lv in ref.levels]
    assert r["level_undecided"] == [lv["undecided"] for lv in ref.levels]
    mask = (1 << pkg.SPLIT_PATH_BITS) - 1
    got = sorted((int(c) & mask, int(t), int(k)) for c, t, k in zip(codes, depth, cls))
    assert got == sorted(ref.leaves)


@pytest.mark.parametrize("name,f,D", CASES[1:])
def test_split_set_is_the_top_of_the_root_scores(pkg, name, f, D):
    p = _shrunk(name, f)
    _, _, _, _, S = _gpu_count(pkg, p, 2)
    assert len(S) == min(16, p.d) and list(S) == sorted(S)
    s = oracle.root_scores(p.net, p.lo, p.hi, p.prop)
    out = np.setdiff1d(np.arange(p.d), S)
    if out.size:
        assert s[S].min() >= s[out].max() * (1 - 1e-4)


def test_split_set_mnist_shaped(pkg):
    """784 inputs: the GPU's set against the oracle's scores of the set and of
    100 sampled dimensions outside it (kinks skipped)."""
    p = gen.make("mnist")
    _, _, _, _, S = _gpu_count(pkg, p, 1)
    assert len(S) == 16
    rng = np.random.default_rng(0)
    out = rng.choice(np.setdiff1d(np.arange(p.d), S), 100, replace=False)
    g = oracle.radius_gradient(p.net, p.lo, p.hi, p.prop, dims=np.concatenate([S, out]))
    w = p.hi.astype(np.float64) - p.lo
    s_in, s_out = np.abs(g[S]) * w[S], np.abs(g[out]) * w[out]
    s_in, s_out = s_in[np.isfinite(s_in)], s_out[np.isfinite(s_out)]
    assert s_in.size >= 12 and s_out.size >= 80
    assert s_in.min() >= s_out.max() * (1 - 1e-4)


@pytest.mark.parametrize("name,f,D", CASES[1:])
def test_choices_are_near_optimal(pkg, name, f, D):
    """At sampled split nodes, the GPU's dimension scores within rounding of the
    best of S under the oracle's FP64 central differences."""
    p = _shrunk(name, f)
    _, codes, depth, _, S = _gpu_count(pkg, p, D)
    m = _split_map(pkg, codes, depth, S)
    rng = np.random.default_rng(1)
    keys = list(m)
    checked = agree = 0
    for idx in rng.choice(len(keys), min(40, len(keys)), replace=False):
        t, path = keys[idx]
        lo, hi = _node_box(p, path, t, m)
        sc = oracle.box_scores(p.net, lo, hi, p.prop, S)
        j = int(np.searchsorted(S, m[(t, path)]))
        if not np.isfinite(sc[j]):
            continue          # a kink at the chosen dimension
        best = np.nanmax(sc)
        checked += 1
        agree += int(sc[j] == best)
        assert sc[j] >= best * (1 - 1e-3) - 1e-12, (t, path, sc, j)
    assert checked >= 10
    assert agree >= 0.8 * checked


def test_gradient_rule_with_optimised_slopes(pkg):
    """With slope steps the choices use the optimised slopes; decided leaves are
    sound (sampled points), the bracket meets the widest-side one, and the
    count repeats exactly."""
    p = _shrunk("acas", 0.1)
    D = 12
    r, codes, depth, cls, S = _gpu_count(pkg, p, D, alpha_steps=10, alpha_lr=0.1, alpha_margin=0.0)
    r2, *_ = _gpu_count(pkg, p, D, alpha_steps=10, alpha_lr=0.1, alpha_margin=0.0)
    assert (r2["unsafe_lo"], r2["unsafe_hi"], r2["boxes"]) == (r["unsafe_lo"], r["unsafe_hi"], r["boxes"])
    assert r["alpha_boxes"] > 0
    assert sum(1 << (D - int(t)) for t in depth) == 1 << D
    m = _split_map(pkg, codes, depth, S)
    mask = (1 << pkg.SPLIT_PATH_BITS) - 1
    rng = np.random.default_rng(2)
    dec = np.nonzero(cls != oracle.UNDECIDED)[0]
    for i in rng.choice(dec, min(300, dec.size), replace=False):
        lo, hi = _node_box(p, int(codes[i]) & mask, int(depth[i]), m)
        x = lo + (hi - lo) * rng.random((32, p.d))
        u = oracle.unsafe_points(p.net, p.prop, x)
        assert u.all() if cls[i] == oracle.UNSAFE else not u.any()
    w = oracle.count(p.net, p.lo, p.hi, p.prop, D)
    assert r["unsafe_lo"] <= w.unsafe_hi and w.unsafe_lo <= r["unsafe_hi"]


def test_gradient_rule_wide_path(pkg):
    """MNIST-shaped (wide path): replayed in the oracle; equal where no leaf is
    left undecided by the widening, else the oracle's bracket lies inside."""
    p = gen.make("mnist")
    D = 5
    r, codes, depth, cls, S = _gpu_count(pkg, p, D)
    m = _split_map(pkg, codes, depth, S)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D, split=_replay(m))
    assert r["unsafe_lo"] <= ref.unsafe_lo <= ref.unsafe_hi <= r["unsafe_hi"]
    if r["tie_leaves"] == 0:
        assert (r["unsafe_lo"], r["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
        assert r["level_boxes"] == [lv["boxes"] for lv in ref.levels]


def test_split_rule_errors(pkg):
    p = gen.make("tiny")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.count(4)
        with pytest.raises(pkg.SlrError, match="ESTATE"):
            c.split_set()
        c.set_options(split_rule=pkg.SPLIT_GRADIENT)
        with pytest.raises(pkg.SlrError, match="EINVAL"):
            c.count(13)
        c.count(6)
        with pytest.raises(pkg.SlrError, match="ESTATE"):
            c.schedule(6)
        with pytest.raises(pkg.SlrError, match="EUNSUPPORTED"):
            c.count_noalloc(6)
        with pytest.raises(pkg.SlrError, match="EUNSUPPORTED"):
            c.count_batch([p], [6])
        with pytest.raises(pkg.SlrError, match="EINVAL"):
            c.set_options(split_rule=2)
        c.set_options(split_rule=pkg.SPLIT_GRADIENT, relax_mode=pkg.RELAX_PAPER_LITERAL)
        with pytest.raises(pkg.SlrError, match="EUNSUPPORTED"):
            c.count(6)


def test_gradient_rule_tensor_core_path_matches(pkg):
    """The tensor-core tile path decodes the per-box split dimensions the same
    way: with its FP32 and FP64 re-checks it gives the FP32 path's count."""
    p = _shrunk("acas", 0.1)
    D = 10
    a, ca, da, ka, Sa = _gpu_count(pkg, p, D)
    b, cb, db, kb, Sb = _gpu_count(pkg, p, D, precision=pkg.PREC_TC_TF32)
    assert list(Sa) == list(Sb)
    assert (a["unsafe_lo"], a["unsafe_hi"], a["boxes"]) == (b["unsafe_lo"], b["unsafe_hi"], b["boxes"])
    assert sorted(zip(ca.tolist(), da.tolist(), ka.tolist())) == sorted(zip(cb.tolist(), db.tolist(), kb.tolist()))
