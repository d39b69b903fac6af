"""Seeded synthetic inputs for the SLR counter (networks, boxes, properties).

This package holds no part of the counting method.  It only draws random
ReLU networks, input boxes and output properties with the shapes of the
paper's benchmarks (Sec. 4, Table 1; Sec. 4.1), so that the FP64 oracle and
the CUDA library can be fed the same inputs.
"""
from .generators import (  # noqa: F401
    Network, Property, Problem, CONFIGS, make, tiny, acas_shaped, nav_shaped,
    linear_2d, single_layer_1d, rare_violation, mc_violation_rate, batched_uneven, mnist_shaped,
)
