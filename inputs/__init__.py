"""Seeded synthetic inputs shared by the FP64 oracle tests and the GPU path's callers.

This package only *generates* inputs: grid random quantum circuits (gate lists with
their matrices), bitstring batches and random complex tensors.  It holds no
tensor-network arithmetic: no contraction, no slicing, no amplitude evaluation.
Both `oracle/` and `paper_2504_09186_gb300/` may import it; neither imports the other.
"""
from .circuits import (  # noqa: F401
    Gate,
    Circuit,
    SQRT_X,
    SQRT_Y,
    SQRT_W,
    fsim,
    couplers,
    grid_circuit,
)
from .batches import (  # noqa: F401
    random_bitstrings,
    subcube_spec,
    subcube_bitstrings,
    random_complex,
    random_labels_perm,
)
