"""GB300 (sm_103a) implementation of the G2LF / V2LF hot path of
"Real-time 3D Visualization of Radiance Fields on Light Field Displays"
(arXiv 2508.18540): splat a radiance field into depth-binned sweeping planes
once, then composite the planes into every light-field view in one pass.

The computation lives in liblf.so (hand-written CUDA kernels behind the C ABI
of include/lf.h); this package is its thin ctypes binding plus the seeded
synthetic input generators.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "api"]
