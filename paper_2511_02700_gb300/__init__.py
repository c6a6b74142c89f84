"""pide2d: GB300 (sm_103a) solver for two-asset European options under a
bivariate Normal Tempered Stable exponential Levy model (arXiv 2511.02700).

The computation lives in the CUDA library libpide2d.so (C ABI in
include/pide2d.h); ``binding`` is its ctypes binding and ``workloads`` holds
the seeded benchmark and test inputs.
"""
