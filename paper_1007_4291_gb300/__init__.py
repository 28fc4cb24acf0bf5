"""GB300-native moving-PML sweeping preconditioner for the 2D Helmholtz equation.

Layout:
  csrc/    CUDA sources of libhs.so (sm_103a): plan and PML tables, batched
           subproblem factorisation, two-front sweep, stencil matvec, FGMRES.
  hs.py    ctypes binding of the C ABI in include/hs.h (marshalling only).
  build.py in-tree nvcc build of libhs.so.
  inputs.py seeded synthetic velocity fields and sources.

Importing the package does not load the CUDA library; ``hs.load()`` does, and
raises if it is missing.
"""
