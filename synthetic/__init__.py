"""Seeded synthetic inputs shared by the GPU path's tests/bench and the oracle.

This package draws random circuits, qubit layouts, bitstrings and random test
tensors. It holds none of the method's arithmetic: no gate matrices, no tensor
network, no contraction. A circuit here is a list of gate *identifiers* and
qubit pairs; each consumer turns identifiers into matrices with its own code.
"""

from .circuits import (  # noqa: F401
    SplitMix64,
    Circuit,
    Layout,
    grid_layout,
    diagonal53_layout,
    random_circuit,
    random_bits,
    random_uniform,
    config_circuit,
    CONFIGS,
)
