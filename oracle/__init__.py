"""FP64 CPU oracle of the NEP hot path -- test infrastructure only.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline use this package.  The CUDA library never imports it.
"""
from .oracle import *  # noqa: F401,F403
