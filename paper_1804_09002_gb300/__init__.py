"""GB300-native Zolo-csd: CS decomposition via two polar decompositions.

The compute path is the CUDA library ``libzolo_csd.so`` (C ABI in
include/zolo_csd.h); ``binding`` is its ctypes front end.  ``inputs`` holds
the seeded synthetic workload generators.  Importing ``binding`` fails loudly
when the library has not been built (``paper_1804_09002_gb300.build``).
"""
__all__ = ["binding", "inputs", "build"]
