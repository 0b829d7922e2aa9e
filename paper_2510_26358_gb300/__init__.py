"""GB300-native multi-view differentiable Gaussian splatting (the mapping and
pose-refinement hot path of AgriGS-SLAM, Sec. III-B and III-C).

The compute path is ``libgsraster.so`` (CUDA for sm_103a, C ABI in
``include/gs.h``); ``gsraster`` is its thin Python binding and ``scenes``
draws seeded synthetic inputs.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "gsraster", "build"]
