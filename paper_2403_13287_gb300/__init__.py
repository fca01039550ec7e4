"""GB300-native (sm_103a) q-LSKUM hot path: CUDA kernels behind a C ABI.

Submodules:
  cloudgen  seeded synthetic NACA 0012 point clouds (inputs only)
  build     nvcc build of the CUDA library (liblskum.so)
  lskum     ctypes binding of include/lskum.h (Solver)
"""
__all__ = ["cloudgen", "build", "lskum"]
