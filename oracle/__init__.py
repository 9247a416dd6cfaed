"""FP64 CPU oracle for occlusion-point reuse.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``, never by the library itself.
"""
from .oracle import *  # noqa: F401,F403
