"""FP64 CPU oracle for Spar-Sink (Li, Yu, Li & Meng, JMLR 2023).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
leg of ``bench.py`` may import this package; the product path (the CUDA
library and its Python binding) never does, and shares no code with it.

The arithmetic lives in ``sparsink_oracle.c`` (plain C, FP64, one function
per step of the paper's algorithms).  This module compiles it with gcc and
exposes thin numpy wrappers.  Citations (paper sections, equations and
algorithms) are in the C file next to each function.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build_oracle, load  # noqa: F401
