"""GB300 (sm_103a) Spar-Sink: importance-sparsified Sinkhorn for OT and UOT.

The compute path is the CUDA library ``libsparsink.so`` behind the C ABI in
``include/sparsink.h``; ``sparsink`` is its thin Python binding and ``inputs``
holds the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "sparsink", "build"]
