"""Seeded synthetic RGB-D input generator (analytic ray casting on the CPU).

This package produces inputs only: depth/colour frames, ground-truth poses and
ground-truth static masks.  It contains none of the reconstruction method's
arithmetic and is shared, as an input producer, by the tests, the oracle runs
and the benchmark.
"""
from .scenes import (  # noqa: F401
    Camera,
    Scene,
    Sequence,
    CONFIGS,
    make_sequence,
    render,
    look_at,
    pose_from_rpy,
)
