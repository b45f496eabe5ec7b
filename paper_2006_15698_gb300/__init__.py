"""GB300-native DG Euler solver: the right-hand side of Kirby & Mavriplis's
collocated Gauss-Legendre discontinuous Galerkin method for the 3D
compressible Euler equations, fused with its low-storage Runge-Kutta update,
as hand-written sm_103a CUDA kernels behind a C ABI (include/dg.h).

Importing the package loads nothing; ``paper_2006_15698_gb300.dg`` loads the
compiled library and raises if it is missing.
"""
__all__ = ["dg", "inputs"]
