"""The oracle's level-by-level count over a pool of host processes (test infrastructure only).

The same breadth-first count as ``counter.count`` (Alg. 1 with a depth cap,
all boxes of a level evaluated together, Sec. 3), with each level's boxes
dealt in chunks to worker processes.  Every box is still bounded by
``slr.slr_forward`` and classified by ``slr.classify`` exactly as there; the
pool only decides which process evaluates which box, so the per-level
statistics, the bracket and the leaf set equal ``counter.count``'s (pinned by
``tests/test_oracle_pins.py``).

Workers are started with the ``spawn`` method: a pool forked after a CUDA
context exists in the parent would hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

_STATE = None
_BLAS_THREADS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _spawn_pool(procs, initializer=None, initargs=()):
    """A spawn pool whose workers run single-threaded BLAS: the variables must be
    in the environment the workers start with (numpy reads them at import)."""
    saved = {v: os.environ.get(v) for v in _BLAS_THREADS}
    for v in _BLAS_THREADS:
        os.environ[v] = "1"
    try:
        return mp.get_context("spawn").Pool(procs, initializer=initializer, initargs=initargs)
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def _init(problem, D):
    global _STATE
    from . import counter
    _STATE = (problem, counter.split_schedule(problem.lo, problem.hi, D), D)


def _level(args):
    codes, t, leaves = args
    from .counter import decode
    from .slr import UNDECIDED, UNSAFE, SAFE, classify, slr_forward
    p, sched, D = _STATE
    codes = np.asarray(codes, dtype=np.int64)
    lo, hi = decode(codes, t, sched, p.lo, p.hi)
    rlo, rhi, _ = slr_forward(p.net, lo, hi, p.prop)
    cls = classify(rlo, rhi, p.prop)
    und = codes[cls == UNDECIDED]
    out = {"undecided": und, "unsafe": int(np.count_nonzero(cls == UNSAFE)),
           "safe": int(np.count_nonzero(cls == SAFE))}
    if leaves:
        keep = (cls != UNDECIDED) if t < D else np.ones(cls.shape[0], dtype=bool)
        out["leaf_codes"] = codes[keep]
        out["leaf_cls"] = cls[keep].astype(np.int8)
    return out


def count_levels(problem, D, procs=None, budget_s=None, leaves=False, chunks_per_proc=4):
    """The oracle's count of ``problem`` to depth D on ``procs`` processes.

    Stops at a level boundary once ``budget_s`` seconds have passed (None: run
    every level).  Returns a dict with the levels evaluated (``levels``: per
    level boxes, safe, unsafe, undecided), ``complete`` (all D + 1 levels, or
    the frontier emptied), the bracket ``unsafe_lo``/``unsafe_hi`` (the
    whole count's when complete), ``boxes``, ``seconds`` (the level loop's
    wall time, without starting the pool) and, with ``leaves``, the leaves as
    arrays ``leaf_codes``, ``leaf_depth``, ``leaf_cls``.
    """
    procs = procs or os.cpu_count() or 1
    levels = []
    lcodes, ldepth, lcls = [], [], []
    with _spawn_pool(procs, _init, (problem, D)) as pool:
        pool.map(_level, [(np.zeros(1, np.int64), 0, False)] * procs)    # start every worker
        frontier = np.zeros(1, dtype=np.int64)
        lo = und_d = 0
        complete = False
        t0 = time.perf_counter()
        for t in range(D + 1):
            if frontier.shape[0] == 0:
                complete = True
                break
            n_chunks = max(1, min(procs * chunks_per_proc, frontier.shape[0]))
            parts = [c for c in np.array_split(frontier, n_chunks) if c.size]
            res = pool.map(_level, [(c, t, leaves) for c in parts])
            und = np.concatenate([r["undecided"] for r in res])
            lv = {"boxes": int(frontier.shape[0]), "safe": sum(r["safe"] for r in res),
                  "unsafe": sum(r["unsafe"] for r in res), "undecided": int(und.shape[0])}
            levels.append(lv)
            lo += lv["unsafe"] << (D - t)
            if leaves:
                for r in res:
                    lcodes.append(r["leaf_codes"])
                    lcls.append(r["leaf_cls"])
                    ldepth.append(np.full(r["leaf_codes"].shape[0], t, dtype=np.int16))
            if t < D:
                frontier = np.concatenate([2 * und, 2 * und + 1])
            else:
                und_d = int(und.shape[0])
                complete = True
            if budget_s is not None and not complete and time.perf_counter() - t0 > budget_s:
                break
        seconds = time.perf_counter() - t0
    out = {"levels": levels, "complete": complete, "unsafe_lo": lo, "unsafe_hi": lo + und_d,
           "boxes": sum(lv["boxes"] for lv in levels), "seconds": seconds, "procs": procs}
    if leaves:
        cat = (lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dtype=dt))
        out["leaf_codes"] = cat(lcodes, np.int64)
        out["leaf_depth"] = cat(ldepth, np.int16)
        out["leaf_cls"] = cat(lcls, np.int8)
    return out


def _fd_part(args):
    from .grad import fd_gradients
    net, lo, hi, prop, alpha, w_hi, w_lo, a_idx, b_idx = args
    return fd_gradients(net, lo, hi, prop, alpha, w_hi, w_lo, w_idx={}, alpha_idx=a_idx, box_idx=b_idx)


def fd_gradients_sampled(net, lo, hi, prop, alpha, w_hi, w_lo, alpha_idx, box_idx, procs=None):
    """``grad.fd_gradients`` at the given slope and box coordinates only (no weights),
    the coordinates dealt over ``procs`` processes; every coordinate is
    differenced exactly as there.  Returns 'alpha' (the concatenated slopes,
    NaN where not differenced or at a kink), 'lo' and 'hi'."""
    procs = procs or os.cpu_count() or 1
    alpha_idx = list(alpha_idx) if alpha is not None else []
    box_idx = list(box_idx)
    jobs = []
    for k in range(procs):
        a, b = alpha_idx[k::procs], box_idx[k::procs]
        if a or b:
            jobs.append((net, lo, hi, prop, alpha, w_hi, w_lo, a, b))
    H = sum(x.size for x in alpha) if alpha is not None else 0
    d = np.asarray(lo).shape[0]
    out = {"alpha": np.full(H, np.nan), "lo": np.full(d, np.nan), "hi": np.full(d, np.nan)}
    with _spawn_pool(min(procs, max(1, len(jobs)))) as pool:
        for r in pool.map(_fd_part, jobs):
            parts = {"alpha": np.concatenate(r["alpha"]) if H else np.zeros(0), "lo": r["lo"], "hi": r["hi"]}
            for key, v in parts.items():
                ok = ~np.isnan(v)
                out[key][ok] = v[ok]
    return out
