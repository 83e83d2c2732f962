"""FP64 CPU oracle for the free-flight expansion (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline legs
may import this package.  It shares no code with the CUDA path.
"""
from .ffx_oracle import *  # noqa: F401,F403
