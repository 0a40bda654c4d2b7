"""GB300 (sm_103a) sliced tensor-network contraction of random-circuit amplitudes.

The compute path lives in libtnc.so (C boundary: include/tnc.h); `tnc` is its ctypes
binding and `autograd` exposes the adjoint contraction to torch.autograd.
"""
from .tnc import (  # noqa: F401
    Context,
    Plan,
    TncError,
    load_library,
    version,
)
