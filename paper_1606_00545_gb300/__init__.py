"""GB300-native ILU(k)/RAS-preconditioned Krylov hot path (Yang, Liu, Chen: Krylov and AMG
linear solvers for large-scale sparse matrices on GPUs).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through :mod:`paper_1606_00545_gb300.hecgpu` (a ctypes binding of the
C ABI in ``include/hecgpu.h``).  :mod:`paper_1606_00545_gb300.synth` holds the
seeded input generators.  Importing the package loads nothing.
"""
