"""Planted mistakes in the oracle's later functions (CPU): the Moore-interval
pass, the finite-difference gradients and their objective, the gradient
split rule's decision weights and radius derivative, the approximate
counter's leaf volume and split side, and the S-shaped relaxation.

Each mutant is the oracle function's own source with one plausible slip (a
dropped clamp, swapped interval ends, a flipped comparison, a dropped factor,
ties to the other end, max for min), compiled in the function's module and
patched in wherever the function is looked up; at least one pin of that
function, each checked against values that do not come from the oracle's
code, must then fail."""
import inspect
import textwrap

import pytest

import oracle
from oracle import approx as oapprox
from oracle import counter as ocnt
from oracle import grad as ograd
from oracle import slr as oslr
from oracle import split as osplit

from . import pins
from . import test_oracle_approx as tapprox
from . import test_oracle_pins as topins
from . import test_oracle_split as tsplit
from . import test_oracle_sshaped as tsshaped


def _mutant(module, name, old, new):
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, (name, old)
    ns = dict(module.__dict__)
    exec(compile(src.replace(old, new), f"<mutant of {module.__name__}.{name}>", "exec"), ns)
    return ns[name]


def _fast_pins(golden):
    def run():
        for _, check in pins.fast_checks(golden):
            check()
    return run


MUTANTS = [
    # (id, module, function, old, new, modules that look the function up, pins)
    ("interval_relu_not_clamped", oslr, "interval_forward",
     "l, u = np.where(l2 > 0, l2, l2 * 0), np.where(u2 > 0, u2, u2 * 0)", "l, u = l2, u2",
     (oracle, oslr, ocnt), "fast"),
    ("interval_ends_swapped", oslr, "interval_forward",
     "l2 = (Wp @ l[..., :, None])[..., 0] + (Wn @ u[..., :, None])[..., 0] + bb",
     "l2 = (Wp @ l[..., :, None])[..., 0] + (Wn @ l[..., :, None])[..., 0] + bb",
     (oracle, oslr, ocnt), "fast"),
    ("decision_direction_flipped", osplit, "decision_weights",
     "if safe_gap <= unsafe_gap:", "if safe_gap > unsafe_gap:",
     (oracle, osplit), tsplit.test_decision_weights_hand_worked),
    ("leaf_volume_drops_a_factor", oapprox, "volume_ratio",
     "for i in range(len(a)):", "for i in range(len(a) - 1):",
     (oapprox,), tapprox.test_leaf_brackets_contain_the_closed_form_area),
    ("split_ties_to_highest_index", oapprox, "widest_side",
     "return int(np.argmax(w)), float(np.max(w))", "return int(len(w) - 1 - np.argmax(w[::-1])), float(np.max(w))",
     (oapprox,), tapprox.test_ties_split_the_lowest_index),
    ("central_difference_over_h", ograd, "_central",
     "g.flat[i] = (f(x0 + e) - f(x0 - e)) / (2 * h)", "g.flat[i] = (f(x0 + e) - f(x0 - e)) / h",
     (ograd,), topins.test_box_gradient_of_an_affine_network_closed_form),
    ("central_difference_sign", ograd, "_central",
     "g.flat[i] = (f(x0 + e) - f(x0 - e)) / (2 * h)", "g.flat[i] = (f(x0 - e) - f(x0 + e)) / (2 * h)",
     (ograd,), topins.test_default_slope_box_gradient_closed_form),
    ("objective_weights_on_the_other_bound", ograd, "objective",
     "np.dot(w_hi, rhi[0]) + np.dot(w_lo, rlo[0])", "np.dot(w_hi, rlo[0]) + np.dot(w_lo, rhi[0])",
     (oracle, ograd, osplit), topins.test_slope_gradient_hand_worked),
    ("radius_stencil_shifts_the_box", osplit, "radius_gradient",
     "objective(net, lo - s * e, hi + s * e, prop, None, w_hi, w_lo)",
     "objective(net, lo + s * e, hi + s * e, prop, None, w_hi, w_lo)",
     (oracle, osplit), lambda: tsplit.test_radius_gradient_of_an_affine_map_is_abs_weight(0)),
    ("straddling_slope_max", oslr, "_relax_s",
     "lam = np.minimum(act_slope(name, l), act_slope(name, u))",
     "lam = np.maximum(act_slope(name, l), act_slope(name, u))",
     (oslr,), tsshaped.test_straddling_interval_uses_the_smaller_end_slope),
]


@pytest.mark.parametrize("mid,module,name,old,new,where,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(monkeypatch, golden, mid, module, name, old, new, where, pin):
    check = _fast_pins(golden) if pin == "fast" else pin
    check()                                            # the pin holds for the oracle as it is
    bad = _mutant(module, name, old, new)
    for m in where:
        if hasattr(m, name):
            monkeypatch.setattr(m, name, bad)
    with pytest.raises(AssertionError):                # a pin fails, not a crash of the mutant
        check()
