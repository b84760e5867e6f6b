"""B300-native implementation of the ATON radiative-transfer step (Aubert & Teyssier 2010).

The product is libaton.so (C ABI in include/aton.h, CUDA kernels for sm_103a in csrc/);
``aton`` is its thin Python binding and ``workloads`` makes seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "aton", "build"]
