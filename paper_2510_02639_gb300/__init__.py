"""GB300-native image-centred ray shooting (ICRS) for microlensing.

The CUDA library (csrc/, C ABI in include/icrs.h) is loaded by the ``icrs``
submodule; importing the package itself loads nothing, so the seeded workload
generators in ``inputs`` can be used without a GPU.
"""
