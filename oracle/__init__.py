"""CPU oracle of the block-decomposed sort (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
