"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each one.

A pin that no mutant can fail would pin nothing; this test shows that a dropped
term, a wrong sign, a swapped operand or a wrong index anywhere in the oracle
breaks at least one of the checks in tests/pins.py.
"""
import numpy as np
import pytest

import oracle
from oracle import counter as ocnt
from oracle import slr as oslr

from . import pins

_orig_concretize = oslr.concretize
_orig_relax = oslr._relax
_orig_fold = oslr.fold_property
_orig_classify = oslr.classify
_orig_sched = ocnt.split_schedule
_orig_decode = ocnt.decode


def _conc_swap(E, a, b):
    lo, hi = _orig_concretize(E, a, b)
    return hi, lo


def _conc_noabs(E, a, b):
    g, g0 = E[..., :-1], E[..., -1]
    m, r = (a + b) / 2, (b - a) / 2
    c = g0 + (g @ m[..., :, None])[..., 0]
    s = (g @ r[..., :, None])[..., 0]
    return c - s, c + s


def _conc_center_at_a(E, a, b):
    g, g0 = E[..., :-1], E[..., -1]
    r = (b - a) / 2
    c = g0 + (g @ a[..., :, None])[..., 0]
    s = (np.abs(g) @ r[..., :, None])[..., 0]
    return c - s, c + s


def _relax_bad_intercept(U, L, ll, ul, lu, uu):
    U2, L2 = _orig_relax(U, L, ll, ul, lu, uu, None, "neurify")
    chord = ~(ll >= 0) & ~(uu <= 0) & (lu < 0)
    s = np.where(chord, uu / np.where(chord, uu - lu, 1.0), 0.0)
    U2[..., -1] = U2[..., -1] + 2 * s * lu          # intercept +s*lu instead of -s*lu
    return U2, L2


def _relax_alpha_from_upper(U, L, ll, ul, lu, uu, alpha, mode):
    unst = ~(ll >= 0) & ~(uu <= 0) & (ul > 0)
    a = np.where(unst, uu / np.where(unst, uu - ll, 1.0), 0.0)
    return _orig_relax(U, L, ll, ul, lu, uu, a, mode)


def _relax_inactive_kept(U, L, ll, ul, lu, uu, alpha, mode):
    U2, L2 = _orig_relax(U, L, ll, ul, lu, uu, alpha, mode)
    inact = ~(ll >= 0) & (uu <= 0)
    U2 = np.where(inact[..., None], U, U2)
    L2 = np.where(inact[..., None], L, L2)
    return U2, L2


def _relax_active_test_wrong(U, L, ll, ul, lu, uu, alpha, mode):
    return _orig_relax(U, L, np.where(ul >= 0, np.abs(ll), ll), ul, lu, uu, alpha, mode)


def _relax_no_lower_zero(U, L, ll, ul, lu, uu, alpha, mode):
    U2, L2 = _orig_relax(U, L, ll, ul, lu, uu, alpha, mode)
    z = ~(ll >= 0) & ~(uu <= 0) & (ul <= 0)
    return U2, np.where(z[..., None], L, L2)


def _fold_drop_e(net, prop):
    Ws, bs = _orig_fold(net, prop)
    if prop is not None:
        bs[-1] = bs[-1] - np.asarray(prop.e)
    return Ws, bs


def _fold_drop_hidden_bias(net, prop):
    Ws, bs = _orig_fold(net, prop)
    return Ws, [b * 0 if k < len(bs) - 1 else b for k, b in enumerate(bs)]


def _fold_transposed(net, prop):
    Ws, bs = _orig_fold(net, prop)
    Ws = [W.T if W.shape[0] == W.shape[1] else W for W in Ws]
    return Ws, bs


def _classify_ignore_strict(lo, hi, prop):
    class P:
        pass
    q = P()
    q.strict = np.zeros_like(np.asarray(prop.strict))
    q.rows_per_clause = prop.rows_per_clause
    return _orig_classify(lo, hi, q)


def _classify_safe_needs_all_rows(lo, hi, prop):
    cls = _orig_classify(lo, hi, prop)
    strict = np.asarray(prop.strict).astype(bool)
    out = np.where(strict, hi <= 0, hi < 0)
    allout = np.all(out, axis=-1)
    cls = np.where((cls == oracle.SAFE) & ~allout, oracle.UNDECIDED, cls).astype(np.int8)
    return cls


def _sched_ties_high(a, b, D):
    w = np.asarray(b, np.float64) - np.asarray(a, np.float64)
    c = np.zeros(w.shape[0], np.int64)
    out = []
    for _ in range(D):
        s = w * np.ldexp(1.0, -c)
        i = int(len(s) - 1 - np.argmax(s[::-1]))
        out.append(i)
        c[i] += 1
    return np.array(out, np.int64)


def _decode_lsb_first(codes, t, sched, a, b):
    codes = np.asarray(codes, np.int64)
    rev = np.zeros_like(codes)
    for j in range(t):
        rev |= ((codes >> j) & 1) << (t - 1 - j)
    return _orig_decode(rev, t, sched, a, b)


def _patch(monkeypatch, name, fn, mods):
    for m in mods:
        if hasattr(m, name):
            monkeypatch.setattr(m, name, fn)


MUTANTS = [
    ("concretize_swapped", "concretize", _conc_swap, (oracle, oslr)),
    ("concretize_no_abs", "concretize", _conc_noabs, (oracle, oslr)),
    ("concretize_centre_at_a", "concretize", _conc_center_at_a, (oracle, oslr)),
    ("chord_intercept_sign", "_relax", lambda *a: _relax_bad_intercept(*a[:6]), (oslr,)),
    ("lower_slope_from_upper_eq", "_relax", _relax_alpha_from_upper, (oslr,)),
    ("inactive_not_zeroed", "_relax", _relax_inactive_kept, (oslr,)),
    ("active_test_wrong", "_relax", _relax_active_test_wrong, (oslr,)),
    ("nonpositive_lower_kept", "_relax", _relax_no_lower_zero, (oslr,)),
    ("property_constant_dropped", "fold_property", _fold_drop_e, (oslr,)),
    ("hidden_bias_dropped", "fold_property", _fold_drop_hidden_bias, (oslr,)),
    ("weights_transposed", "fold_property", _fold_transposed, (oslr,)),
    ("strictness_ignored", "classify", _classify_ignore_strict, (oracle, oslr, ocnt)),
    ("safe_needs_every_row", "classify", _classify_safe_needs_all_rows, (oracle, oslr, ocnt)),
    ("ties_to_highest_index", "split_schedule", _sched_ties_high, (oracle, ocnt)),
    ("path_bits_lsb_first", "decode", _decode_lsb_first, (oracle, ocnt)),
]


@pytest.mark.parametrize("mname,attr,fn,mods", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(monkeypatch, golden, mname, attr, fn, mods):
    _patch(monkeypatch, attr, fn, mods)
    caught = []
    for cname, check in pins.fast_checks(golden):
        try:
            check()
        except Exception:  # noqa: BLE001 - any failure counts as caught
            caught.append(cname)
            break
    assert caught, f"mutant {mname} passed every pin"
