"""GB300 (sm_103a) directional scale-discretized wavelet transform on the sphere.

The compute path is libs2dw.so (hand-written CUDA behind the C ABI of
include/s2dw.h); ``binding`` is its ctypes binding.  ``inputs`` holds the
seeded synthetic-input generators.
"""
__all__ = ["binding", "inputs"]
