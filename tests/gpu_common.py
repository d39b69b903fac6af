"""Helpers shared by the GPU tests: tolerances and leaf checks against the oracle."""
from __future__ import annotations

import numpy as np

import oracle

# Bounds agree with the FP64 oracle within this fraction of the row's scale
# max(|lo|, |hi|) + (hi - lo): FP32 rounding plus the outward widening.
BOUND_RTOL = 1e-5


def bound_errors(gpu_lo, gpu_hi, o_lo, o_hi):
    scale = np.maximum(np.abs(o_lo), np.abs(o_hi)) + (o_hi - o_lo) + 1e-30
    return np.abs(gpu_lo - o_lo) / scale, np.abs(gpu_hi - o_hi) / scale, scale


def random_sub_boxes(p, n, seed, min_frac=0.0):
    rng = np.random.default_rng(seed)
    u = np.sort(rng.random((2, n, p.d)), axis=0)
    if min_frac > 0:
        u[1] = np.maximum(u[1], np.minimum(u[0] + min_frac, 1.0))
    lo = (p.lo + (p.hi - p.lo) * u[0]).astype(np.float32)
    hi = (p.lo + (p.hi - p.lo) * u[1]).astype(np.float32)
    return lo, hi


def oracle_classes_of(p, codes, depth, D):
    """Oracle classes of boxes given by (code, depth) pairs under the depth-D schedule."""
    sched = oracle.split_schedule(p.lo, p.hi, D)
    out = np.empty(len(codes), dtype=np.int8)
    codes = np.asarray(codes, dtype=np.int64)
    depth = np.asarray(depth)
    for t in np.unique(depth):
        sel = np.nonzero(depth == t)[0]
        lo, hi = oracle.decode(codes[sel], int(t), sched, p.lo, p.hi)
        rlo, rhi, _ = oracle.slr_forward(p.net, lo, hi, p.prop)
        out[sel] = oracle.classify(rlo, rhi, p.prop)
    return out


def leaves_partition_root(codes, depth, D):
    """Sum of 2^(D-t) over leaves equals 2^D exactly (the leaves tile the root box)."""
    return int(sum(1 << (D - int(t)) for t in depth)) == 1 << D
