"""Plain FP64 CPU oracle of the rail-based KMC step (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.
"""
from .oracle import *  # noqa: F401,F403
