"""Seeded generators for the synthetic workloads.

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) in one
fixed order: W_1, b_1, ..., W_K, b_K, then the input box, then the property.
Weights follow He initialisation, N(0, 2/fan_in) (variance), biases
N(0, 0.1) (variance).  All arrays are float32: the network, box and property
that both the oracle and the CUDA path analyse are these float32 values.

The property is the *unsafe* set (the negation of the postcondition Q,
Sec. 3): a disjunction over clauses of a conjunction of linear rows
``C[r] . y + e[r] >= 0`` (``> 0`` where ``strict[r]``).

The only arithmetic here is a plain forward pass used to pick seeds whose
Monte-Carlo violation rate lies in a window (so that a workload is neither
trivially safe nor trivially unsafe); it is not part of the counting method.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    """K affine layers; an activation after every layer but the last.

    ``W[k]`` has shape (widths[k+1], widths[k]); ``b[k]`` has widths[k+1].
    ``act[k]`` names the activation after layer k ('relu', 'tanh' or
    'sigmoid'); an empty list means ReLU everywhere.
    """
    W: list
    b: list
    act: list = field(default_factory=list)

    def activation(self, k):
        return self.act[k] if self.act else "relu"

    @property
    def widths(self):
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]

    @property
    def K(self):
        return len(self.W)


@dataclass
class Property:
    """Unsafe set: OR over clauses of AND over rows of C[r].y + e[r] >= 0 (> 0 if strict)."""
    rows_per_clause: np.ndarray  # int32 (n_clauses,)
    C: np.ndarray                # float32 (R, n_out)
    e: np.ndarray                # float32 (R,)
    strict: np.ndarray           # uint8 (R,)

    @property
    def R(self):
        return int(self.C.shape[0])


@dataclass
class Problem:
    name: str
    net: Network
    lo: np.ndarray   # float32 (d,)
    hi: np.ndarray   # float32 (d,)
    prop: Property
    depth: int
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def d(self):
        return int(self.lo.shape[0])


def _mlp(rng, widths, bias_var=0.1):
    W, b = [], []
    for k in range(len(widths) - 1):
        fan_in, fan_out = widths[k], widths[k + 1]
        W.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=(fan_out, fan_in)).astype(np.float32))
        b.append(rng.normal(0.0, np.sqrt(bias_var), size=(fan_out,)).astype(np.float32))
    return Network(W, b)


def _prop(clauses):
    """clauses: list of lists of (c_vector, e, strict)."""
    rows = [r for cl in clauses for r in cl]
    return Property(
        rows_per_clause=np.array([len(cl) for cl in clauses], dtype=np.int32),
        C=np.array([r[0] for r in rows], dtype=np.float32).reshape(len(rows), -1),
        e=np.array([r[1] for r in rows], dtype=np.float32),
        strict=np.array([1 if r[2] else 0 for r in rows], dtype=np.uint8),
    )


def _unit(n, i, scale=1.0):
    v = np.zeros(n, dtype=np.float32)
    v[i] = scale
    return v


# ---------------------------------------------------------------------------
# Seed selection (plain forward pass; not the method)
# ---------------------------------------------------------------------------

def _activate(name, h):
    if name == "tanh":
        return np.tanh(h)
    if name == "sigmoid":
        return 1.0 / (1.0 + np.exp(-h))
    return np.maximum(h, 0.0)


def _forward(net, x):
    h = x.astype(np.float32)
    for k in range(net.K):
        h = h @ net.W[k].T + net.b[k]
        if k < net.K - 1:
            h = _activate(net.activation(k), h)
    return h


def _unsafe(prop, y):
    vals = y @ prop.C.T + prop.e
    sat = np.where(prop.strict.astype(bool), vals > 0, vals >= 0)
    out = np.zeros(y.shape[0], dtype=bool)
    r0 = 0
    for nr in prop.rows_per_clause:
        out |= np.all(sat[:, r0:r0 + nr], axis=1)
        r0 += nr
    return out


def mc_violation_rate(p: Problem, n_samples: int, seed: int = 12345) -> float:
    """Fraction of uniform samples of the box that fall in the unsafe set."""
    rng = np.random.default_rng(seed)
    x = p.lo + (p.hi - p.lo) * rng.random((n_samples, p.d), dtype=np.float32)
    return float(np.mean(_unsafe(p.prop, _forward(p.net, x))))


def _first_in_window(gen, base_seed, window, max_tries=4000):
    lo_w, hi_w = window
    for s in range(base_seed, base_seed + max_tries):
        p = gen(s)
        if not (lo_w * 0.5 <= mc_violation_rate(p, 1 << 12, seed=s) <= min(1.0, hi_w * 1.5)):
            continue
        if lo_w <= mc_violation_rate(p, 1 << 16, seed=s) <= hi_w:
            return p
    raise RuntimeError(f"no seed in [{base_seed}, {base_seed + max_tries}) meets VR window {window}")


# ---------------------------------------------------------------------------
# Paper-shaped workloads
# ---------------------------------------------------------------------------

def _tiny_raw(seed):
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [2, 8, 8, 1])
    lo = np.full(2, -1.0, dtype=np.float32)
    hi = np.full(2, 1.0, dtype=np.float32)
    prop = _prop([[(_unit(1, 0, -1.0), 0.0, True)]])          # unsafe: y < 0
    return Problem("tiny_2-8-8-1", net, lo, hi, prop, 16, seed)


def _acas_raw(seed):
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [5] + [50] * 6 + [5])
    side = rng.uniform(0.05, 0.3, size=5)
    a = rng.uniform(-0.5, 0.5 - side)
    lo = a.astype(np.float32)
    hi = (a + side).astype(np.float32)
    # unsafe: output 0 is not minimal, i.e. OR_j (y_0 - y_j > 0)
    clauses = [[(_unit(5, 0) - _unit(5, j), 0.0, True)] for j in range(1, 5)]
    return Problem("acas_5-50x6-5", net, lo, hi, _prop(clauses), 20, seed)


def _nav_raw(seed):
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [22, 64, 64, 3])
    c_lidar = rng.uniform(0.025, 0.975, size=20)
    c_hd = rng.uniform(-0.995, 0.995, size=2)
    lo = np.concatenate([c_lidar - 0.025, c_hd - 0.005]).astype(np.float32)
    hi = np.concatenate([c_lidar + 0.025, c_hd + 0.005]).astype(np.float32)
    # unsafe: action 1 is argmax, y_1 - y_0 >= 0 and y_1 - y_2 >= 0
    prop = _prop([[(_unit(3, 1) - _unit(3, 0), 0.0, False),
                   (_unit(3, 1) - _unit(3, 2), 0.0, False)]])
    return Problem("nav_22-64-64-3", net, lo, hi, prop, 24, seed)


def _mnist_raw(seed, radius=0.02):
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [784, 256, 256, 256, 10])
    x0 = rng.random(784)
    lo = np.clip(x0 - radius, 0.0, 1.0).astype(np.float32)
    hi = np.clip(x0 + radius, 0.0, 1.0).astype(np.float32)
    # unsafe: class 0 is not the argmax, OR_j (y_j - y_0 >= 0)
    clauses = [[(_unit(10, j) - _unit(10, 0), 0.0, False)] for j in range(1, 10)]
    p = Problem("mnist_784-256x3-10", net, lo, hi, _prop(clauses), 12, seed)
    p.extra["centre"] = x0.astype(np.float32)
    return p


@functools.lru_cache(maxsize=64)
def tiny(seed: int = 0) -> Problem:
    """2 -> 8 -> 8 -> 1 on [-1,1]^2, unsafe y < 0, depth 16; VR in [5%, 95%]."""
    return _first_in_window(_tiny_raw, seed, (0.05, 0.95))


@functools.lru_cache(maxsize=64)
def acas_shaped(seed: int = 0) -> Problem:
    """5 -> 6x50 -> 5 (ACAS Xu shape, Sec. 4), 4 clauses y_0 > y_j, depth 20; VR in [0.5%, 50%]."""
    return _first_in_window(_acas_raw, seed, (0.005, 0.5))


@functools.lru_cache(maxsize=64)
def nav_shaped(seed: int = 0) -> Problem:
    """22 -> 64 -> 64 -> 3 (mapless-navigation shape, Sec. 4), action 1 argmax, depth 24; VR in [5%, 50%]."""
    return _first_in_window(_nav_raw, seed, (0.05, 0.5))


@functools.lru_cache(maxsize=16)
def mnist_shaped(seed: int = 0) -> Problem:
    """784 -> 3x256 -> 10 (an MNIST-classifier shape), L-inf ball of radius 0.02 around a
    random point of [0,1]^784 clipped to [0,1], class 0 stays argmax, depth 12.  The
    first seed at or above `seed` whose network puts class 0 on top at the centre."""
    for s in range(seed, seed + 1000):
        p = _mnist_raw(s)
        if int(np.argmax(_forward(p.net, p.extra["centre"][None])[0])) == 0:
            return p
    raise RuntimeError("no seed puts class 0 on top")


def _acas_tanh_raw(seed):
    p = _acas_raw(seed)
    p.net.act = ["tanh"] * (p.net.K - 1)
    p.name = "acas_tanh_5-50x6-5"
    return p


def _nav_sigmoid_raw(seed):
    p = _nav_raw(seed)
    p.net.act = ["sigmoid"] * (p.net.K - 1)
    p.name = "nav_sigmoid_22-64-64-3"
    return p


def _tiny_act_raw(act):
    def raw(seed):
        p = _tiny_raw(seed)
        p.net.act = [act] * (p.net.K - 1)
        p.name = f"tiny_{act}_2-8-8-1"
        return p
    return raw


@functools.lru_cache(maxsize=16)
def tiny_tanh(seed: int = 0) -> Problem:
    """The tiny workload with tanh after both hidden layers; VR in [5%, 95%]."""
    return _first_in_window(_tiny_act_raw("tanh"), seed, (0.05, 0.95))


@functools.lru_cache(maxsize=16)
def tiny_sigmoid(seed: int = 0) -> Problem:
    """The tiny workload with the logistic sigmoid after both hidden layers; VR in [5%, 95%]."""
    return _first_in_window(_tiny_act_raw("sigmoid"), seed, (0.05, 0.95))


@functools.lru_cache(maxsize=16)
def acas_tanh(seed: int = 0) -> Problem:
    """The ACAS-shaped workload with tanh after every hidden layer (Sec. 3 names other
    activations as an extension of the ReLU relaxation); VR in [0.5%, 50%]."""
    return _first_in_window(_acas_tanh_raw, seed, (0.005, 0.5))


@functools.lru_cache(maxsize=16)
def nav_sigmoid(seed: int = 0) -> Problem:
    """The nav-shaped workload with the logistic sigmoid after every hidden layer; VR in [5%, 50%]."""
    return _first_in_window(_nav_sigmoid_raw, seed, (0.05, 0.5))


def linear_2d(seed: int = 0, depth: int = 12) -> Problem:
    """A single affine layer y = w.x + c on [-1,1]^2, unsafe y < 0 (closed-form test case)."""
    rng = np.random.default_rng(seed)
    W = rng.normal(0.0, 1.0, size=(1, 2)).astype(np.float32)
    b = rng.uniform(-0.5, 0.5, size=(1,)).astype(np.float32)
    net = Network([W], [b])
    lo = np.full(2, -1.0, dtype=np.float32)
    hi = np.full(2, 1.0, dtype=np.float32)
    prop = _prop([[(_unit(1, 0, -1.0), 0.0, True)]])
    return Problem("linear_2d", net, lo, hi, prop, depth, seed)


def single_layer_1d(seed: int = 0, hidden: int = 6, depth: int = 14) -> Problem:
    """1 -> hidden -> 1 on [-1,1], unsafe y < 0 (closed-form test case)."""
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [1, hidden, 1])
    lo = np.array([-1.0], dtype=np.float32)
    hi = np.array([1.0], dtype=np.float32)
    prop = _prop([[(_unit(1, 0, -1.0), 0.0, True)]])
    return Problem("single_layer_1d", net, lo, hi, prop, depth, seed)


def rare_violation(seed: int = 0, depth: int = 18, target_margin: float = 2e-3) -> Problem:
    """3 -> 32 -> 32 -> 1 on [0,1]^3 with Q: y >= 0 (Sec. 4.1).

    The paper gives no weights; the output bias is shifted so that the
    minimum of y over a dense sample grid sits just below zero
    (``-target_margin``), which leaves a tiny unsafe region.
    """
    rng = np.random.default_rng(seed)
    net = _mlp(rng, [3, 32, 32, 1])
    lo = np.zeros(3, dtype=np.float32)
    hi = np.ones(3, dtype=np.float32)
    g = np.linspace(0.0, 1.0, 65, dtype=np.float32)
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ymin = float(_forward(net, grid).min())
    net.b[-1] = (net.b[-1] - np.float32(ymin) - np.float32(target_margin)).astype(np.float32)
    prop = _prop([[(_unit(1, 0, -1.0), 0.0, True)]])          # unsafe: y < 0
    return Problem("rare_3-32-32-1", net, lo, hi, prop, depth, seed)


def _batch_member(rng, d, width, hidden, n_props, depth_range, seed):
    net = _mlp(rng, [d] + [width] * hidden + [int(rng.integers(2, 9))])
    n_out = net.widths[-1]
    out = []
    tries = 0
    while len(out) < n_props and tries < 50 * n_props:
        tries += 1
        side = rng.uniform(0.02, 0.2, size=d)
        a = rng.uniform(-0.5, 0.5 - side)
        lo = a.astype(np.float32)
        hi = (a + side).astype(np.float32)
        rows = []
        for _ in range(int(rng.integers(1, 3))):
            i, j = rng.choice(n_out, size=2, replace=False)
            c = np.zeros(n_out, dtype=np.float32)
            c[i] = rng.uniform(0.5, 2.0)
            c[j] = -rng.uniform(0.5, 2.0)
            rows.append((c, float(rng.normal(0.0, np.sqrt(0.1))), False))
        D = int(rng.integers(depth_range[0], depth_range[1] + 1))
        p = Problem(f"batch_d{d}_w{width}_h{hidden}", net, lo, hi, _prop([rows]), D, seed)
        vr = mc_violation_rate(p, 1 << 12, seed=seed + tries)
        if 0.01 <= vr <= 0.99:
            out.append(p)
    return out


def batched_uneven(seed: int = 0, n_nets: int = 16, props_per_net: int = 16, depth_range=(12, 22),
                   widths=(32, 64, 128), tile_only=True):
    """Many (network, property) problems of uneven size (the batched workload).

    16 seeded networks with inputs d in {5, 8, 16, 32}, hidden widths from
    `widths` and 2-8 hidden layers, each carrying 16 random boxes (sides
    U(0.02, 0.2) inside [-0.5, 0.5]^d) with a one-clause property of 1-2 rows
    a y_i - a' y_j + e >= 0 (a, a' ~ U(0.5, 2), e ~ N(0, 0.1)), redrawn until
    the Monte-Carlo violation rate lies in [1 %, 99 %], and a depth cap
    D ~ U{12..22}.  With `tile_only` a width is kept only when its
    contraction tiles fit the fused kernel, (2d + 3) * width / 8 <= 512;
    otherwise wider networks run on the wide path inside the same call.
    """
    rng = np.random.default_rng(seed)
    probs = []
    ds = [5, 8, 16, 32]
    for k in range(n_nets):
        d = ds[k % len(ds)]
        ok_w = [w for w in widths if not tile_only or (2 * d + 3) * ((w + 7) // 8) <= 512]
        width = int(rng.choice(ok_w))
        hidden = int(rng.integers(2, 9))
        probs += _batch_member(rng, d, width, hidden, props_per_net, depth_range, seed * 1000 + k)
    return probs


CONFIGS = {
    "tiny": tiny,
    "acas": acas_shaped,
    "nav": nav_shaped,
    "mnist": mnist_shaped,
    "rare": rare_violation,
    "acas_tanh": acas_tanh,
    "tiny_tanh": tiny_tanh,
    "tiny_sigmoid": tiny_sigmoid,
    "nav_sigmoid": nav_sigmoid,
}


def make(name: str, seed: int = 0) -> Problem:
    return CONFIGS[name](seed)
