"""GB300-native occlusion-point reuse (ray-traced AO and area-light shadows).

The compute path lives in liboccreuse.so (hand-written sm_103a CUDA behind the C ABI
of include/occ.h); ``paper_2607_23122_gb300.occ`` is its Python binding.
"""
from .build import build  # noqa: F401

__all__ = ["build"]
