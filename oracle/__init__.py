"""FP64 CPU oracle for the exact #DNN-Verification counter (SLR + bisection).

TEST INFRASTRUCTURE ONLY.  Nothing in the library path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may use it.  It shares no code with the CUDA path and follows the
paper's steps one box at a time (NumPy batches over boxes change no box's
arithmetic), in float64, or in exact rationals (``fractions.Fraction``) for
tiny cases.

Modules
  slr      symbolic linear relaxation (Sec. 2.2, Eq. 1; Sec. 3), Moore intervals,
           property fold and classification (Sec. 3 containment check).
  counter  split schedule, path-code decoding and the level-by-level exact
           count (Alg. 1 with a depth cap; Sec. 3 level-parallel BaB).
  grad     central finite differences of the row bounds with respect to the
           lower ReLU slopes, the box, the weights and the biases.
  split    the gradient split rule (a split dimension per box from the
           decision loss's radius gradient).

Every function here is pinned by tests that do not re-use its own formulas
(brute force over box vertices, closed forms, hand-worked examples, sampling).
"""
from .slr import (  # noqa: F401
    SAFE, UNSAFE, UNDECIDED, concretize, interval_forward, slr_forward,
    fold_property, classify, forward_points, unsafe_points, to_exact,
)
from .counter import split_schedule, decode, count, CountResult  # noqa: F401
from .grad import objective, fd_gradients, default_alpha  # noqa: F401
from .split import (  # noqa: F401
    decision_weights, radius_gradient, split_set, root_scores, box_scores, gradient_split,
)
