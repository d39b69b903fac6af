"""Lower-slope optimisation through the C ABI (needs a GB300): slopes in the
sound evaluation, the adjoint against FP64 central differences of the oracle,
projected Adam, and the count with optimised slopes."""
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
    if opt:
        c.set_options(**opt)
    return c


def _split_alpha(net, a):
    """(H,) -> per-hidden-layer list."""
    out, o = [], 0
    for w in net.W[:-1]:
        out.append(a[o:o + w.shape[0]])
        o += w.shape[0]
    return out


def _oracle_bounds_at(p, lo, hi, alpha):
    al = [np.clip(x, 0.0, 1.0).astype(np.float64) for x in _split_alpha_batch(p.net, alpha)]
    return oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop, alpha=al)[:2]


def _split_alpha_batch(net, A):
    out, o = [], 0
    for w in net.W[:-1]:
        out.append(A[:, o:o + w.shape[0]])
        o += w.shape[0]
    return out


# ---------------------------------------------------------------------------
# slopes in the sound evaluation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "acas", "nav"])
@pytest.mark.parametrize("n", [1, 37, 700])
def test_bounds_at_given_slopes_match_oracle(pkg, name, n):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, n, seed=n + 5)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        rng = np.random.default_rng(n)
        A = rng.uniform(-0.2, 1.2, size=(n, H)).astype(np.float32)   # clamped to [0, 1] by the library
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True, alpha=A)
    olo, ohi = _oracle_bounds_at(p, lo, hi, A)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL, (elo.max(), ehi.max())
    ocls = oracle.classify(olo, ohi, p.prop)
    dec = cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], ocls[dec])


def test_nan_slopes_read_as_zero(pkg):
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 64, seed=3)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        A = np.full((64, H), np.nan, dtype=np.float32)
        r1 = c.bounds(lo, hi, alpha=A)
        r2 = c.bounds(lo, hi, alpha=np.zeros((64, H), np.float32))
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


# ---------------------------------------------------------------------------
# the adjoint against FP64 central differences (h = 1e-3) of the oracle
# ---------------------------------------------------------------------------

def _fd_case(p, seed, shrink, free):
    rng = np.random.default_rng(seed)
    lo, hi = random_sub_boxes(p, 1, seed=seed)
    hi = (lo + (hi - lo) / shrink).astype(np.float32)
    R = p.prop.C.shape[0]
    g_lo = rng.normal(size=R)
    g_hi = rng.normal(size=R)
    H = sum(w.shape[0] for w in p.net.W[:-1])
    A = rng.uniform(0.05, 0.95, size=H).astype(np.float32) if free else None
    return lo, hi, g_lo, g_hi, A


def _close(gpu, fd, rtol):
    """gpu vs fd where fd is not a kink (NaN), relative to the array's scale."""
    ok = ~np.isnan(fd)
    if not ok.any():
        return True, 0.0
    scale = max(np.abs(fd[ok]).max(), 1e-3)
    err = np.abs(gpu[ok] - fd[ok]).max() / scale
    return err <= rtol, err


@pytest.mark.parametrize("name,shrink,seeds", [("tiny", 1, range(4)), ("acas", 8, range(3)), ("nav", 4, range(2))])
@pytest.mark.parametrize("free", [True, False])
def test_adjoint_matches_central_differences(pkg, name, shrink, seeds, free):
    p = gen.make(name)
    for seed in seeds:
        lo, hi, g_lo, g_hi, A = _fd_case(p, 100 + seed, shrink, free)
        rng = np.random.default_rng(seed)
        w_idx = None
        if name != "tiny":
            w_idx = {k: rng.choice(w.size, size=min(w.size, 12), replace=False) for k, w in enumerate(p.net.W)}
        fd = oracle.fd_gradients(p.net, lo[0], hi[0], p.prop,
                                 _split_alpha(p.net, A.astype(np.float64)) if free else None,
                                 g_hi, g_lo, w_idx=w_idx)
        with _counter(pkg, p) as c:
            out = c.margin_backward(lo, hi, g_lo[None].astype(np.float32), g_hi[None].astype(np.float32),
                                    alpha=None if A is None else A[None], weights=True)
        rtol = 2e-3
        if free:
            ok, e = _close(out["d_alpha"][0], np.concatenate(fd["alpha"]), rtol)
            assert ok, ("alpha", seed, e)
        for key in ("lo", "hi"):
            ok, e = _close(out["d_" + key][0], fd[key], rtol)
            assert ok, (key, seed, e)
        for k in range(len(p.net.W)):
            ok, e = _close(out["d_W"][k], fd["W"][k], rtol)
            assert ok, ("W", k, seed, e)
            ok, e = _close(out["d_b"][k], fd["b"][k], rtol)
            assert ok, ("b", k, seed, e)


def test_adjoint_row_bounds_and_batch_sum(pkg):
    """The adjoint's own row bounds are the SLR bounds; weight gradients sum over the boxes."""
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 300, seed=9)
    R = p.prop.C.shape[0]
    rng = np.random.default_rng(1)
    g_lo = rng.normal(size=(300, R)).astype(np.float32)
    g_hi = rng.normal(size=(300, R)).astype(np.float32)
    with _counter(pkg, p) as c:
        all_ = c.margin_backward(lo, hi, g_lo, g_hi, weights=True)
        parts = [c.margin_backward(lo[i:i + 100], hi[i:i + 100], g_lo[i:i + 100], g_hi[i:i + 100], weights=True)
                 for i in (0, 100, 200)]
    olo, ohi, _ = oracle.slr_forward(p.net, lo.astype(np.float64), hi.astype(np.float64), p.prop)
    elo, ehi, _ = bound_errors(all_["row_lo"].astype(np.float64), all_["row_hi"].astype(np.float64), olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL
    for k in range(len(p.net.W)):
        s = sum(q["d_W"][k].astype(np.float64) for q in parts)
        scale = np.abs(s).max() + 1e-6
        assert np.abs(all_["d_W"][k] - s).max() <= 1e-4 * scale
    assert np.array_equal(np.concatenate([q["d_alpha"] for q in parts]), all_["d_alpha"])


# ---------------------------------------------------------------------------
# projected Adam on the slopes
# ---------------------------------------------------------------------------

def _undecided_boxes(p, n, depth, seed):
    """Sub-boxes of the depth-`depth` bisection that the default slopes leave UNDECIDED."""
    sched = oracle.split_schedule(p.lo, p.hi, depth)
    rng = np.random.default_rng(seed)
    codes = rng.integers(0, 1 << depth, size=8 * n)
    lo, hi = oracle.decode(codes, depth, sched, p.lo, p.hi)
    rlo, rhi, _ = oracle.slr_forward(p.net, lo, hi, p.prop)
    und = oracle.classify(rlo, rhi, p.prop) == oracle.UNDECIDED
    return lo[und][:n].astype(np.float32), hi[und][:n].astype(np.float32)


@pytest.mark.parametrize("name,depth", [("acas", 12), ("nav", 10), ("tiny", 8)])
def test_optimised_slopes_are_sound_and_no_looser(pkg, name, depth):
    p = gen.make(name)
    lo, hi = _undecided_boxes(p, 200, depth, seed=depth)
    assert len(lo) > 10
    with _counter(pkg, p) as c:
        d_lo, d_hi, d_cls = c.bounds(lo, hi)
        rl, rh, cls, A = c.optimize_alpha(lo, hi, steps=20, lr=0.1)
        al, ah, _, aerr = c.bounds(lo, hi, want_err=True, alpha=A)
    # intersected bounds never looser than the starting slopes'
    assert np.all(rl >= d_lo) and np.all(rh <= d_hi)
    # no looser than the bounds at the final slopes either
    assert np.all(rl >= al) and np.all(rh <= ah)
    # the final slopes' bounds agree with the oracle at those slopes
    olo, ohi = _oracle_bounds_at(p, lo, hi, A)
    assert np.all(al <= olo + 1e-12 * np.abs(olo)) and np.all(ah >= ohi - 1e-12 * np.abs(ohi))
    elo, ehi, _ = bound_errors(al.astype(np.float64) + aerr, ah.astype(np.float64) - aerr, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL
    # slopes stay in [0, 1]
    assert np.all((A >= 0) & (A <= 1))
    # sound: sampled points of every box fall inside the intersected bounds
    rng = np.random.default_rng(0)
    for b in range(len(lo)):
        x = lo[b] + (hi[b] - lo[b]) * rng.random((256, p.d))
        y = oracle.forward_points(p.net, x, p.prop)[0]
        assert np.all(y >= rl[b] - 1e-5 * (1 + np.abs(rl[b]))) and np.all(y <= rh[b] + 1e-5 * (1 + np.abs(rh[b])))
    # the class follows from the intersected bounds
    ocls = oracle.classify(rl.astype(np.float64), rh.astype(np.float64), p.prop)
    assert np.array_equal(cls, ocls)
    # a decided default class stays decided the same way
    dec = d_cls != oracle.UNDECIDED
    assert np.array_equal(cls[dec], d_cls[dec])


def test_optimised_slopes_tighten_acas(pkg):
    p = gen.make("acas")
    lo, hi = _undecided_boxes(p, 256, 14, seed=1)
    with _counter(pkg, p) as c:
        d_lo, d_hi, _ = c.bounds(lo, hi)
        rl, rh, cls, _ = c.optimize_alpha(lo, hi, steps=20, lr=0.1)
    gain = ((rl - d_lo) + (d_hi - rh)).sum()
    assert gain > 0


# ---------------------------------------------------------------------------
# the count with optimised slopes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,D", [("tiny", 14), ("acas", 12), ("nav", 10)])
@pytest.mark.parametrize("margin", [0.0, 0.2])
def test_count_with_slopes_nests_in_fixed_count(pkg, name, D, margin):
    """Every undecided box optimised (margin 0) or only those near a decision
    (margin 0.2, the default): the count nests inside the fixed-slope one,
    which equals the oracle's, and repeats exactly."""
    p = gen.make(name)
    with _counter(pkg, p) as c:
        fixed = c.count(D)
        c.set_options(alpha_steps=20, alpha_lr=0.1, alpha_margin=margin)
        opt = c.count(D)
        again = c.count(D)
        c.set_options(alpha_steps=20, alpha_lr=0.1, alpha_margin=0.0)
        full = c.count(D)
    ref = oracle.count(p.net, p.lo, p.hi, p.prop, D)
    assert (fixed["unsafe_lo"], fixed["unsafe_hi"]) == (ref.unsafe_lo, ref.unsafe_hi)
    assert fixed["unsafe_lo"] <= opt["unsafe_lo"] <= opt["unsafe_hi"] <= fixed["unsafe_hi"]
    assert opt["boxes"] <= fixed["boxes"]
    assert opt["alpha_boxes"] <= full["alpha_boxes"]
    if margin == 0.0:
        assert opt["alpha_boxes"] > 0
    # the optimisation is deterministic: no atomics feed the slopes
    assert (again["unsafe_lo"], again["unsafe_hi"], again["boxes"]) == (opt["unsafe_lo"], opt["unsafe_hi"], opt["boxes"])


# ---------------------------------------------------------------------------
# torch.autograd.Function
# ---------------------------------------------------------------------------

def test_autograd_function(pkg):
    import torch
    from paper_2312_05890_gb300.autograd import SLRRowBounds
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 16, seed=4)
    dev = torch.device("cuda:0")
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        tlo = torch.tensor(lo, device=dev, requires_grad=True)
        thi = torch.tensor(hi, device=dev, requires_grad=True)
        A = torch.full((16, H), 0.5, device=dev, requires_grad=True)
        W = [torch.tensor(w, device=dev, requires_grad=True) for w in p.net.W]
        b = [torch.tensor(x, device=dev, requires_grad=True) for x in p.net.b]
        rlo, rhi = SLRRowBounds.apply(c, tlo, thi, A, *W, *b)
        loss = rhi.sum() - 0.5 * rlo.sum()
        loss.backward()
        R = rlo.shape[1]
        ref = c.margin_backward(lo, hi, np.full((16, R), -0.5, np.float32), np.ones((16, R), np.float32),
                                alpha=np.full((16, H), 0.5, np.float32), weights=True)
    assert np.allclose(rlo.detach().cpu().numpy(), ref["row_lo"]) and np.allclose(rhi.detach().cpu().numpy(), ref["row_hi"])
    assert np.allclose(tlo.grad.cpu().numpy(), ref["d_lo"], rtol=1e-5, atol=1e-6)
    assert np.allclose(A.grad.cpu().numpy(), ref["d_alpha"], rtol=1e-5, atol=1e-6)
    for k in range(len(W)):
        assert np.allclose(W[k].grad.cpu().numpy(), ref["d_W"][k], rtol=1e-4, atol=1e-4)


# ---------------------------------------------------------------------------
# slopes on the wide path (per-box state in GPU memory; adjoint state in
# global memory)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "acas"])
def test_wide_bounds_at_given_slopes(pkg, name):
    p = gen.make(name)
    lo, hi = random_sub_boxes(p, 200, seed=21)
    with _counter(pkg, p, wide=1) as c:
        H = c.alpha_width()
        A = np.random.default_rng(2).uniform(0, 1, size=(200, H)).astype(np.float32)
        rl, rh, cls, err = c.bounds(lo, hi, want_err=True, alpha=A)
    olo, ohi = _oracle_bounds_at(p, lo, hi, A)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(rl <= olo + 1e-12 * scale) and np.all(rh >= ohi - 1e-12 * scale)
    elo, ehi, _ = bound_errors(rl.astype(np.float64) + err, rh.astype(np.float64) - err, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL


@pytest.mark.parametrize("free", [True, False])
def test_wide_adjoint_matches_tile_adjoint(pkg, free):
    """The global-memory adjoint (wide path) computes what the shared-memory one does."""
    p = gen.make("acas")
    lo, hi = random_sub_boxes(p, 64, seed=8)
    R = p.prop.C.shape[0]
    rng = np.random.default_rng(3)
    g_lo = rng.normal(size=(64, R)).astype(np.float32)
    g_hi = rng.normal(size=(64, R)).astype(np.float32)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        A = rng.uniform(0.05, 0.95, size=(64, H)).astype(np.float32) if free else None
        a = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A, weights=True)
    with _counter(pkg, p, wide=1) as c:
        b = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A, weights=True)
    for key in ("row_lo", "row_hi", "d_lo", "d_hi") + (("d_alpha",) if free else ()):
        assert np.array_equal(a[key], b[key]), key
    # weight gradients are sums over boxes in a different grouping and atomic order
    for k in range(len(p.net.W)):
        scale = np.abs(a["d_W"][k]).max() + 1e-6
        assert np.abs(a["d_W"][k] - b["d_W"][k]).max() <= 1e-5 * scale


def _boxes_differing(a, b, keys, n, rtol):
    """Boxes where some array of `keys` differs by more than rtol of that box's scale."""
    bad = set()
    for key in keys:
        x = np.asarray(a[key], np.float64).reshape(n, -1)
        y = np.asarray(b[key], np.float64).reshape(n, -1)
        scale = np.abs(x).max(axis=1, keepdims=True) + 1e-6
        bad |= set(np.nonzero((np.abs(x - y) / scale).max(axis=1) > rtol)[0].tolist())
    return bad


@pytest.mark.parametrize("free", [True, False])
def test_wide_product_adjoint_matches_tile_adjoint(pkg, free):
    """Without weight gradients the wide path runs the adjoint as per-layer
    tensor-core products (three-term TF32); it agrees with the one-box kernel
    to float rounding (at most one box may sit on a ReLU case boundary that
    the two summation orders resolve differently)."""
    p = gen.make("acas")
    n = 64
    lo, hi = random_sub_boxes(p, n, seed=9)
    R = p.prop.C.shape[0]
    rng = np.random.default_rng(4)
    g_lo = rng.normal(size=(n, R)).astype(np.float32)
    g_hi = rng.normal(size=(n, R)).astype(np.float32)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        A = rng.uniform(0.05, 0.95, size=(n, H)).astype(np.float32) if free else None
        a = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A)
    with _counter(pkg, p, wide=1) as c:
        b = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A)
    keys = ("row_lo", "row_hi", "d_lo", "d_hi") + (("d_alpha",) if free else ())
    assert len(_boxes_differing(a, b, keys, n, 1e-4)) <= 1


def test_wide_product_adjoint_mnist_shaped(pkg):
    """784 -> 3x256 -> 10: the per-layer product adjoint against the one-box
    global-memory kernel (which the weight gradients select), slopes free and
    default."""
    p = gen.make("mnist")
    n = 6
    lo, hi = random_sub_boxes(p, n, seed=6, min_frac=0.5)
    R = p.prop.C.shape[0]
    rng = np.random.default_rng(5)
    g_lo = rng.normal(size=(n, R)).astype(np.float32)
    g_hi = rng.normal(size=(n, R)).astype(np.float32)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        for A in (None, rng.uniform(0.05, 0.95, size=(n, H)).astype(np.float32)):
            fast = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A)
            slow = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A, weights=True)
            keys = ("row_lo", "row_hi", "d_lo", "d_hi") + (("d_alpha",) if A is not None else ())
            assert len(_boxes_differing(fast, slow, keys, n, 1e-4)) <= 1


def test_wide_slopes_mnist_shaped(pkg):
    """784 -> 3x256 -> 10: optimised slopes give sound bounds no looser than the default."""
    p = gen.make("mnist")
    lo, hi = random_sub_boxes(p, 6, seed=5, min_frac=0.5)
    with _counter(pkg, p) as c:
        d_lo, d_hi, _ = c.bounds(lo, hi)
        rl, rh, cls, A = c.optimize_alpha(lo, hi, steps=5, lr=0.1)
        al, ah, _, aerr = c.bounds(lo, hi, want_err=True, alpha=A)
    assert np.all(rl >= d_lo) and np.all(rh <= d_hi)
    assert np.all(rl >= al) and np.all(rh <= ah)
    olo, ohi = _oracle_bounds_at(p, lo, hi, A)
    scale = np.maximum(np.abs(olo), np.abs(ohi)) + (ohi - olo)
    assert np.all(al <= olo + 1e-12 * scale) and np.all(ah >= ohi - 1e-12 * scale)
    elo, ehi, _ = bound_errors(al.astype(np.float64) + aerr, ah.astype(np.float64) - aerr, olo, ohi)
    assert elo.max() <= BOUND_RTOL and ehi.max() <= BOUND_RTOL
    rng = np.random.default_rng(0)
    for b in range(len(lo)):
        x = lo[b] + (hi[b] - lo[b]) * rng.random((500, p.d))
        y = oracle.forward_points(p.net, x, p.prop)[0]
        assert np.all(y >= rl[b]) and np.all(y <= rh[b])


def test_wide_count_with_slopes_nests(pkg):
    p = gen.make("acas")
    D = 11
    with _counter(pkg, p, wide=1) as c:
        fixed = c.count(D)
        c.set_options(wide=1, alpha_steps=10, alpha_lr=0.1, alpha_margin=0.0)
        opt = c.count(D)
    assert fixed["unsafe_lo"] <= opt["unsafe_lo"] <= opt["unsafe_hi"] <= fixed["unsafe_hi"]
    assert opt["alpha_boxes"] > 0


@pytest.mark.parametrize("free", [True, False])
def test_wide_product_adjoint_mnist_against_oracle(pkg, free):
    """784 -> 3x256 -> 10: the per-layer tensor-core product adjoint that the
    slope-optimised MNIST-shaped count runs, against the FP64 oracle's central
    differences (h = 1e-3) at 200 sampled slope coordinates and 100 sampled
    input dimensions (both endpoints) of each of two boxes, within 2e-3 of each
    array's scale; free slopes and the default slopes u/(u-l)."""
    from oracle import pool
    p = gen.make("mnist")
    n = 2
    lo, hi = random_sub_boxes(p, n, seed=16, min_frac=0.5)
    R = p.prop.C.shape[0]
    rng = np.random.default_rng(21 + int(free))
    g_lo = rng.normal(size=(n, R)).astype(np.float32)
    g_hi = rng.normal(size=(n, R)).astype(np.float32)
    with _counter(pkg, p) as c:
        H = c.alpha_width()
        A = rng.uniform(0.05, 0.95, size=(n, H)).astype(np.float32) if free else None
        out = c.margin_backward(lo, hi, g_lo, g_hi, alpha=A)
    checked = 0
    for b in range(n):
        a_idx = sorted(rng.choice(H, size=200, replace=False).tolist())
        b_idx = sorted(rng.choice(p.d, size=100, replace=False).tolist())
        fd = pool.fd_gradients_sampled(p.net, lo[b].astype(np.float64), hi[b].astype(np.float64), p.prop,
                                       _split_alpha(p.net, A[b].astype(np.float64)) if free else None,
                                       g_hi[b].astype(np.float64), g_lo[b].astype(np.float64), a_idx, b_idx)
        pairs = [("d_lo", "lo"), ("d_hi", "hi")] + ([("d_alpha", "alpha")] if free else [])
        for gkey, fkey in pairs:
            ok, e = _close(out[gkey][b], fd[fkey], 2e-3)
            assert ok, (gkey, b, e)
            checked += int(np.count_nonzero(~np.isnan(fd[fkey])))
    # a quarter of the coordinates at least is kink-free (a box side is 0.02-0.04
    # wide, so h = 1e-3 flips some neuron's case for about half the box coordinates)
    assert checked >= (n * (200 + 2 * 100) if free else n * 2 * 100) // 4
