"""FP64 CPU oracle of the micro-edge rasterizer-gradient method (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does.
"""
from .oracle import *  # noqa: F401,F403
