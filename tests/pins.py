"""Checks that pin the FP64 oracle to facts outside itself.

Each check raises AssertionError when the oracle disagrees with:
  * brute force (box vertices, dense samples, grids),
  * closed forms (affine regions, a 1-D piecewise-linear net, a 2-D linear net),
  * hand-worked examples (tests/golden/hand_worked.json).
None of them re-types the oracle's own formulas.  They are shared by the pin
tests and by the mutation test, which plants mistakes in the oracle and
expects at least one check to fail.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle
from oracle import slr as oslr
from workloads import generators as gen

CLS = {"SAFE": oracle.SAFE, "UNSAFE": oracle.UNSAFE, "UNDECIDED": oracle.UNDECIDED}


def _net(W, b):
    return gen.Network([np.array(w, dtype=np.float32) for w in W],
                       [np.array(x, dtype=np.float32) for x in b])


def _vertices(lo, hi):
    d = len(lo)
    return np.array([[hi[i] if (v >> i) & 1 else lo[i] for i in range(d)]
                     for v in range(1 << d)], dtype=np.float64)


# ---------------------------------------------------------------------------
# concretisation vs the 2^d box vertices
# ---------------------------------------------------------------------------

def check_concretize_vertices(seed=0):
    rng = np.random.default_rng(seed)
    for d in (1, 2, 3, 5, 8):
        E = rng.normal(size=(7, d + 1))
        a = rng.uniform(-2, 1, size=d)
        b = a + rng.uniform(0, 2, size=d)
        lo, hi = oracle.concretize(E, a, b)
        V = _vertices(a, b)
        vals = V @ E[:, :-1].T + E[:, -1]
        np.testing.assert_allclose(lo, vals.min(0), rtol=0, atol=1e-12)
        np.testing.assert_allclose(hi, vals.max(0), rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# hand-worked examples
# ---------------------------------------------------------------------------

def check_hand_bounds(golden):
    for ex in golden["bounds"]:
        net = _net(ex["W"], ex["b"])
        a = np.array(ex["box_lo"])
        b = np.array(ex["box_hi"])
        for mode in ("neurify", "paper_literal"):
            lo, hi, pre = oracle.slr_forward(net, a, b, None, mode=mode)
            np.testing.assert_allclose(lo, ex[mode][0], atol=1e-15, err_msg=f"{ex['name']} {mode} lo")
            np.testing.assert_allclose(hi, ex[mode][1], atol=1e-15, err_msg=f"{ex['name']} {mode} hi")
            if "pre" in ex and mode == "neurify":
                for k, want in enumerate(ex["pre"]):
                    for got, w in zip(pre[k], want):
                        np.testing.assert_allclose(got, w, atol=1e-15, err_msg=f"{ex['name']} pre {k}")
        lo, hi, _ = oracle.interval_forward(net, a, b, None)
        np.testing.assert_allclose(lo, ex["interval"][0], atol=1e-15)
        np.testing.assert_allclose(hi, ex["interval"][1], atol=1e-15)


def check_hand_classify(golden):
    g = golden["classify"]
    for case in g["cases"]:
        prop = gen.Property(np.array(g["rows_per_clause"], np.int32),
                            np.zeros((3, 1), np.float32), np.zeros(3, np.float32),
                            np.array(case["strict"], np.uint8))
        got = oracle.classify(np.array(case["lo"]), np.array(case["hi"]), prop)
        assert int(got) == CLS[case["class"]], case


def check_hand_schedule(golden):
    g = golden["schedule"]
    s = oracle.split_schedule(np.array(g["box_lo"], np.float32), np.array(g["box_hi"], np.float32), g["depth"])
    assert s.tolist() == g["sched"], s
    dc = g["decode"]
    lo, hi = oracle.decode(np.array([dc["code"]]), dc["t"], s, g["box_lo"], g["box_hi"])
    assert lo[0].tolist() == dc["lo"] and hi[0].tolist() == dc["hi"], (lo, hi)


def check_hand_count(golden):
    for ex in golden["count"]:
        net = _net(ex["W"], ex["b"])
        prop = gen.Property(np.array(ex["rows_per_clause"], np.int32), np.array(ex["C"], np.float32),
                            np.array(ex["e"], np.float32), np.array(ex["strict"], np.uint8))
        r = oracle.count(net, np.array(ex["box_lo"], np.float32), np.array(ex["box_hi"], np.float32),
                         prop, ex["depth"])
        assert (r.unsafe_lo, r.unsafe_hi) == (ex["unsafe_lo"], ex["unsafe_hi"]), (ex["name"], r.unsafe_lo, r.unsafe_hi)
        got = [[lv["boxes"], lv["safe"], lv["unsafe"], lv["undecided"]] for lv in r.levels]
        assert got == ex["levels"], (ex["name"], got)


# ---------------------------------------------------------------------------
# SLR is exact where no ReLU is unstable: compare with the composed affine map
# ---------------------------------------------------------------------------

def check_exact_on_stable_region(seed=0, n_cases=12):
    rng = np.random.default_rng(seed)
    shapes = [[2, 8, 8, 1], [5, 12, 12, 12, 4], [3, 6, 2]]
    done = 0
    tries = 0
    while done < n_cases and tries < 4000:
        tries += 1
        widths = shapes[done % len(shapes)]
        net = gen._mlp(rng, widths)
        x0 = rng.uniform(-1, 1, size=widths[0])
        # activation pattern and composed affine map at x0 (plain matrix products)
        J = np.eye(widths[0])
        c = np.zeros(widths[0])
        h = x0.copy()
        margin = np.inf
        for k in range(net.K):
            W = net.W[k].astype(np.float64)
            bb = net.b[k].astype(np.float64)
            z = W @ h + bb
            J, c = W @ J, W @ c + bb
            if k < net.K - 1:
                act = (z > 0).astype(np.float64)
                margin = min(margin, float(np.min(np.abs(z))))
                h = z * act
                J, c = act[:, None] * J, act * c
        rad = 0.2 * margin / (1e-9 + np.abs(J).sum(axis=1).max() + 50.0)
        # a box small enough that no pre-activation changes sign on it
        r = rng.uniform(0.3, 1.0, size=widths[0]) * rad
        a, b = x0 - r, x0 + r
        lo, hi, pre = oracle.slr_forward(net, a, b, None)
        # every hidden neuron must be stable for this check to apply
        stable = all(np.all((p[0] >= 0) | (p[3] <= 0)) for p in pre)
        if not stable:
            continue
        V = _vertices(a, b)
        vals = V @ J.T + c
        scale = np.abs(vals).max() + 1.0
        np.testing.assert_allclose(lo, vals.min(0), rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(hi, vals.max(0), rtol=0, atol=1e-12 * scale)
        done += 1
    assert done == n_cases, f"only {done} stable cases found"


def check_affine_net_exact(seed=0):
    """A network with no ReLU (one affine layer) is bounded exactly."""
    rng = np.random.default_rng(seed)
    for d in (1, 2, 4, 6):
        W = rng.normal(size=(3, d)).astype(np.float32)
        b = rng.normal(size=(3,)).astype(np.float32)
        net = gen.Network([W], [b])
        a = rng.uniform(-1, 0, size=d)
        bb = a + rng.uniform(0.1, 1, size=d)
        lo, hi, _ = oracle.slr_forward(net, a, bb, None)
        vals = _vertices(a, bb) @ W.astype(np.float64).T + b
        np.testing.assert_allclose(lo, vals.min(0), atol=1e-12)
        np.testing.assert_allclose(hi, vals.max(0), atol=1e-12)


# ---------------------------------------------------------------------------
# soundness: sampled points and grids lie inside the bounds
# ---------------------------------------------------------------------------

def _sub_boxes(rng, lo, hi, n):
    lo = lo.astype(np.float64)
    hi = hi.astype(np.float64)
    out = [(lo, hi)]
    for _ in range(n):
        u = np.sort(rng.uniform(0, 1, size=(2, lo.shape[0])), axis=0)
        out.append((lo + (hi - lo) * u[0], lo + (hi - lo) * u[1]))
    return out


def check_soundness_sampling(problems, n_points=20000, n_boxes=6, seed=0, mode="neurify"):
    rng = np.random.default_rng(seed)
    for p in problems:
        for a, b in _sub_boxes(rng, p.lo, p.hi, n_boxes):
            lo, hi, pre = oracle.slr_forward(p.net, a, b, p.prop, mode=mode)
            x = a + (b - a) * rng.random((n_points, a.shape[0]))
            if a.shape[0] <= 8:
                x = np.concatenate([x, _vertices(a, b)])
            rows, zs = oracle.forward_points(p.net, x, p.prop)
            tol = 1e-9 * (1.0 + np.abs(rows).max())
            assert np.all(rows >= lo - tol) and np.all(rows <= hi + tol), (p.name, mode)
            for (ll, ul, lu, uu), z in zip(pre, zs):
                t = 1e-9 * (1.0 + np.abs(z).max())
                assert np.all(z >= ll - t) and np.all(z <= uu + t), (p.name, "hidden")
                assert np.all(ll <= ul + t) and np.all(lu <= uu + t)


def check_grid_2d(problem, n=256):
    g0 = np.linspace(problem.lo[0], problem.hi[0], n)
    g1 = np.linspace(problem.lo[1], problem.hi[1], n)
    x = np.stack(np.meshgrid(g0, g1, indexing="ij"), -1).reshape(-1, 2)
    lo, hi, _ = oracle.slr_forward(problem.net, problem.lo, problem.hi, problem.prop)
    rows, _ = oracle.forward_points(problem.net, x, problem.prop)
    assert np.all(rows >= lo - 1e-9) and np.all(rows <= hi + 1e-9)


# ---------------------------------------------------------------------------
# counts vs closed forms
# ---------------------------------------------------------------------------

def _halfplane_area(w, c, lo, hi):
    """Area of {x in box : w.x + c < 0} by clipping the box polygon (Sutherland-Hodgman)."""
    poly = [(lo[0], lo[1]), (hi[0], lo[1]), (hi[0], hi[1]), (lo[0], hi[1])]
    f = lambda q: w[0] * q[0] + w[1] * q[1] + c  # noqa: E731
    out = []
    for i in range(len(poly)):
        p, q = poly[i], poly[(i + 1) % len(poly)]
        fp, fq = f(p), f(q)
        if fp < 0:
            out.append(p)
        if (fp < 0) != (fq < 0):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    if len(out) < 3:
        return 0.0
    s = 0.0
    for i in range(len(out)):
        x1, y1 = out[i]
        x2, y2 = out[(i + 1) % len(out)]
        s += x1 * y2 - x2 * y1
    return abs(s) / 2


def check_count_linear_2d(seeds=(0, 1, 2, 3), depth=10):
    for s in seeds:
        p = gen.linear_2d(s, depth)
        r = oracle.count(p.net, p.lo, p.hi, p.prop, depth)
        # brute force over the 2^(D/2) x 2^(D/2) grid cells: unsafe iff every corner has y < 0
        n = 1 << (depth // 2)
        g = np.linspace(-1.0, 1.0, n + 1)
        w = p.net.W[0][0].astype(np.float64)
        c = float(p.net.b[0][0])
        Y = w[0] * g[:, None] + w[1] * g[None, :] + c
        corners = np.stack([Y[:-1, :-1], Y[1:, :-1], Y[:-1, 1:], Y[1:, 1:]])
        all_uns = np.all(corners < 0, axis=0)
        all_safe = np.all(corners >= 0, axis=0)
        assert r.unsafe_lo == int(all_uns.sum()), (s, r.unsafe_lo, int(all_uns.sum()))
        assert r.unsafe_hi - r.unsafe_lo == int((~all_uns & ~all_safe).sum())
        area = _halfplane_area(w, c, (-1.0, -1.0), (1.0, 1.0)) / 4.0
        assert r.unsafe_lo / 2 ** depth <= area + 1e-12 <= r.unsafe_hi / 2 ** depth + 2e-12


def _pwl_unsafe_length(net, a, b):
    """Exact measure of {x in [a,b] : y(x) < 0} for a 1 -> h -> 1 ReLU net."""
    w1 = net.W[0][:, 0].astype(np.float64)
    b1 = net.b[0].astype(np.float64)
    w2 = net.W[1][0].astype(np.float64)
    b2 = float(net.b[1][0])
    bps = sorted({a, b} | {float(-bb / ww) for ww, bb in zip(w1, b1) if ww != 0 and a < -bb / ww < b})
    y = lambda x: float(w2 @ np.maximum(w1 * x + b1, 0.0) + b2)  # noqa: E731
    length = 0.0
    n_roots = 0
    for x0, x1 in zip(bps[:-1], bps[1:]):
        y0, y1 = y(x0), y(x1)
        if y0 < 0 and y1 < 0:
            length += x1 - x0
        elif y0 < 0 <= y1 or y1 < 0 <= y0:
            xr = x0 + (x1 - x0) * y0 / (y0 - y1)
            n_roots += 1
            length += (xr - x0) if y0 < 0 else (x1 - xr)
    return length, n_roots, len(bps) - 2


def check_count_1d(seeds=(0, 1, 2, 3, 4, 5), depth=14):
    for s in seeds:
        p = gen.single_layer_1d(s, depth=depth)
        r = oracle.count(p.net, p.lo, p.hi, p.prop, depth)
        length, n_roots, n_bp = _pwl_unsafe_length(p.net, -1.0, 1.0)
        frac = length / 2.0
        assert r.unsafe_lo / 2 ** depth <= frac + 1e-12, (s, r.unsafe_lo, frac)
        assert frac <= r.unsafe_hi / 2 ** depth + 1e-12, (s, r.unsafe_hi, frac)
        assert r.unsafe_hi - r.unsafe_lo <= 2 * n_roots + 2 * n_bp + 2, (s, r.unsafe_lo, r.unsafe_hi, n_roots, n_bp)


def check_leaves_by_sampling(problem, depth, n_per_leaf=64, seed=0):
    rng = np.random.default_rng(seed)
    r = oracle.count(problem.net, problem.lo, problem.hi, problem.prop, depth, collect_leaves=True)
    sched = oracle.split_schedule(problem.lo, problem.hi, depth)
    for cls in (oracle.SAFE, oracle.UNSAFE):
        sel = [(c, t) for c, t, k in r.leaves if k == cls]
        for c, t in sel[:200]:
            lo, hi = oracle.decode(np.array([c]), t, sched, problem.lo, problem.hi)
            x = lo + (hi - lo) * rng.random((n_per_leaf, lo.shape[1]))
            uns = oracle.unsafe_points(problem.net, problem.prop, x)
            assert np.all(uns) if cls == oracle.UNSAFE else not np.any(uns), (c, t, cls)
    return r


ALL_FAST = None  # filled by the mutation test


def with_offsets(p, seed=0):
    """A copy of problem p whose property rows carry non-zero constants e."""
    import copy
    q = copy.deepcopy(p)
    rng = np.random.default_rng(seed)
    q.prop.e = rng.normal(0.0, 0.3, size=q.prop.e.shape).astype(np.float32)
    q.name = p.name + "+e"
    return q


def fast_checks(golden):
    """The quick pins, as (name, thunk) pairs, for the mutation test."""
    return [
        ("concretize_vertices", lambda: check_concretize_vertices()),
        ("hand_bounds", lambda: check_hand_bounds(golden)),
        ("hand_classify", lambda: check_hand_classify(golden)),
        ("hand_schedule", lambda: check_hand_schedule(golden)),
        ("hand_count", lambda: check_hand_count(golden)),
        ("stable_region", lambda: check_exact_on_stable_region(n_cases=4)),
        ("affine_exact", lambda: check_affine_net_exact()),
        ("soundness", lambda: check_soundness_sampling(
            [gen.tiny(0), with_offsets(gen.acas_shaped(0))], n_points=4000, n_boxes=3)),
        ("linear_2d", lambda: check_count_linear_2d(seeds=(0, 1), depth=8)),
        ("count_1d", lambda: check_count_1d(seeds=(0, 1, 2), depth=10)),
    ]
