"""CPU FP64 oracle of the nonlinear-reconstruction solve (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
