"""GB300-native (sm_103a) ReFusion per-frame hot path.

The compute lives in ``librefusion.so`` (CUDA, C ABI in ``include/refusion.h``);
``refusion`` is its thin Python binding and ``build`` compiles it in-tree.
"""
from . import build  # noqa: F401

__all__ = ["build", "refusion"]
