"""FP64 CPU oracle of the tensorial Chebyshev method (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package. The CUDA library never calls it.
"""
from .oracle import *  # noqa: F401,F403
