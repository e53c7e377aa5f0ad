"""GB300-native batched B-spline projection and inversion (arXiv 2504.11498).

Submodules:
  bspl   -- ctypes binding of libbspl.so (include/bspl.h); loads the CUDA
            library on first use and raises if it is missing.
  build  -- nvcc build of libbspl.so for sm_103a.
  synth  -- seeded synthetic workloads (inputs only).
"""
