"""B300-native SENSE / unrolled-reconstruction hot path (Blumenthal et al.,
"Deep, Deep Learning with BART").

The compute runs in libsense.so (hand-written CUDA for sm_103a, C ABI in
include/sense.h); the Python modules only marshal torch tensors into it.
Importing this package does not load the library; the first call does, and
raises if it is missing.
"""
__all__ = ["SensePlan"]


def __getattr__(name):
    if name == "SensePlan":
        from .sense import SensePlan
        return SensePlan
    raise AttributeError(name)
